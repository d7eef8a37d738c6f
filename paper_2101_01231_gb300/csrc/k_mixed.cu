// Mixed-precision prediction (placeholder until the tensor-core kernel lands).
#include "ridg_internal.h"
namespace ridg {
bool mixed_supported(int, int, int) { return false; }
int mixed_build(int, int, const std::vector<double>&, int, int, std::vector<unsigned short>&,
                std::vector<double>&, MixedOp&) { return RIDG_EINVAL; }
cudaError_t launch_predict_mixed(const Grid&, int, const double*, const MixedOp&, double*, int,
                                 int*, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace ridg
