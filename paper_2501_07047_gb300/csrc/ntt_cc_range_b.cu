// Instantiations of the CUDA-core NTT kernels for log2 N in {12, 13, 14}.
#include "ntt_cc_impl.cuh"

namespace hefx {
namespace cc {

cudaError_t launch_range_b(int logn, NttMode mode, const KArgs& a, size_t rows, cudaStream_t s, bool lazy) {
    switch (logn) {
        case 12: return launch_mode<12>(mode, a, rows, s, lazy);
        case 13: return launch_mode<13>(mode, a, rows, s, lazy);
        case 14: return launch_mode<14>(mode, a, rows, s, lazy);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cc
}  // namespace hefx
