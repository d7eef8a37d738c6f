// The batched Burgers ensemble's Newton prediction in one launch over every degree's region
// queue (FP32 block solves); a translation unit of its own so that it compiles beside the others.
#include "k_newton.cuh"

namespace ridg {
cudaError_t launch_newton_multi_f32(const NewtonMulti& m, const NewtonMulti* dev, int grid,
                                 cudaStream_t s) {
  return newton::launch_multi_typed<float, false>(m, dev, grid, s);
}
int newton_multi_ctas_per_sm_f32() { return newton::multi_ctas_per_sm<float, false>(); }
}  // namespace ridg
