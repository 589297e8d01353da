// Tensor-core basis conversion -- under construction.
#include "bconv_common.h"

namespace hefx {
cudaError_t bconv_tc_upload(hefx_bconv_plan*, const BConvConst&) { return cudaSuccess; }
void bconv_tc_free(hefx_bconv_plan*) {}
bool bconv_tc_available(const hefx_bconv_plan*) { return false; }
cudaError_t launch_bconv_tc(const hefx_bconv_plan*, const uint32_t*, uint32_t*, size_t, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace hefx
