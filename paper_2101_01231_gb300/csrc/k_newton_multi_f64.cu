// The batched Burgers ensemble's Newton prediction in one launch over every degree's region
// queue (FP64 block solves); a translation unit of its own so that it compiles beside the others.
#include "k_newton.cuh"

namespace ridg {
cudaError_t launch_newton_multi_f64(const NewtonMulti& m, const NewtonMulti* dev, int grid,
                                 cudaStream_t s) {
  return newton::launch_multi_typed<double, false>(m, dev, grid, s);
}
int newton_multi_ctas_per_sm_f64() { return newton::multi_ctas_per_sm<double, false>(); }
}  // namespace ridg
