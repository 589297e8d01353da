// Instantiations of the CUDA-core NTT kernels for log2 N in {16}.
#include "ntt_cc_impl.cuh"

namespace hefx {
namespace cc {

cudaError_t launch_range_d(int logn, NttMode mode, const KArgs& a, size_t rows, cudaStream_t s, bool lazy) {
    switch (logn) {
        case 16: return launch_mode<16>(mode, a, rows, s, lazy);
        default: return cudaErrorInvalidValue;
    }
}

int max_clusters_16(NttMode mode, bool lazy) {
    if (mode == MODE_FWD) return lazy ? max_active_clusters<16, MODE_FWD, 2>() : max_active_clusters<16, MODE_FWD, 0>();
    if (mode == MODE_INV) return lazy ? max_active_clusters<16, MODE_INV, 2>() : max_active_clusters<16, MODE_INV, 0>();
    return 0;
}

}  // namespace cc
}  // namespace hefx
