// Instantiations of the CUDA-core NTT kernels for log2 N in {17}.
#include "ntt_cc_impl.cuh"

namespace hefx {
namespace cc {

cudaError_t launch_range_e(int logn, NttMode mode, const KArgs& a, size_t rows, cudaStream_t s, bool lazy) {
    switch (logn) {
        case 17: return launch_mode<17>(mode, a, rows, s, lazy);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cc
}  // namespace hefx
