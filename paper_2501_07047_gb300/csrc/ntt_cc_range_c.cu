// Instantiations of the CUDA-core NTT kernels for log2 N in {15}.
#include "ntt_cc_impl.cuh"

namespace hefx {
namespace cc {

cudaError_t launch_range_c(int logn, NttMode mode, const KArgs& a, size_t rows, cudaStream_t s, bool lazy) {
    switch (logn) {
        case 15: return launch_mode<15>(mode, a, rows, s, lazy);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cc
}  // namespace hefx
