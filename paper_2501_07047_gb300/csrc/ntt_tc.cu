// Tensor-core (tcgen05) layout-invariant matrix NTT -- under construction.
#include "hefx_internal.h"

namespace hefx {
bool tc_supported(const hefx_params*) { return false; }
cudaError_t tc_prepare(hefx_params*) { return cudaErrorNotSupported; }
void tc_free(hefx_params*) {}
cudaError_t launch_ntt_tc(const hefx_params*, NttMode, const uint32_t*, const uint32_t*, uint32_t*, size_t,
                          cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace hefx
