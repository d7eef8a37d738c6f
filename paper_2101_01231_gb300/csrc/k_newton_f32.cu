// Newton prediction with FP32 linear solves and the FP64 residual (RIDG_PREC_MIXED_FP32):
// the factorisation only steers the iteration, the FP64 residual fixes the converged point.
#include "k_newton.cuh"

namespace ridg {
cudaError_t launch_newton_f32(int nb, int m, int kind, const NewtonArgs& a, int grid,
                              cudaStream_t s) {
  return newton::launch_typed<float, false>(nb, m, kind, a, grid, s);
}
int newton_ctas_per_sm_f32(int nb, int m, int kind) { return newton::ctas_per_sm<float, false>(nb, m, kind); }
}  // namespace ridg
