// Newton prediction with FP64 linear solves (RIDG_PREC_FP64).
#include "k_newton.cuh"

namespace ridg {
cudaError_t launch_newton_f64(int nb, int m, int kind, const NewtonArgs& a, int grid,
                              cudaStream_t s) {
  return newton::launch_typed<double, false>(nb, m, kind, a, grid, s);
}
int newton_ctas_per_sm_f64(int nb, int m, int kind) { return newton::ctas_per_sm<double, false>(nb, m, kind); }
}  // namespace ridg
