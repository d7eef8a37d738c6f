// Newton prediction with FP64 linear solves (RIDG_PREC_FP64).
#include "k_newton.cuh"

namespace ridg {
cudaError_t launch_newton_f64(int nb, int m, int kind, const NewtonArgs& a, int grid,
                              cudaStream_t s) {
  return newton::launch_typed<double>(nb, m, kind, a, grid, s);
}
}  // namespace ridg
