// Newton prediction with the Schur-complement block updates on the TF32 tensor cores
// (RIDG_PREC_MIXED_TF32): tcgen05.mma kind::tf32 with FP32 accumulation, FP32 pivot inverses,
// and refinement sweeps against the FP64 residual, which fixes the converged point.
#include "k_newton.cuh"

namespace ridg {
cudaError_t launch_newton_tf32(int nb, int m, int kind, const NewtonArgs& a, int grid,
                               cudaStream_t s) {
  return newton::launch_typed<float, true>(nb, m, kind, a, grid, s);
}
int newton_ctas_per_sm_tf32(int nb, int m, int kind) {
  return newton::ctas_per_sm<float, true>(nb, m, kind);
}
}  // namespace ridg
