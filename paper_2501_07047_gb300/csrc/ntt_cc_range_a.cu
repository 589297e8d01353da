// Instantiations of the CUDA-core NTT kernels for log2 N in {3, 4, 5, 6, 7, 8, 9, 10, 11}.
#include "ntt_cc_impl.cuh"

namespace hefx {
namespace cc {

cudaError_t launch_range_a(int logn, NttMode mode, const KArgs& a, size_t rows, cudaStream_t s, bool lazy) {
    switch (logn) {
        case 3: return launch_mode<3>(mode, a, rows, s, lazy);
        case 4: return launch_mode<4>(mode, a, rows, s, lazy);
        case 5: return launch_mode<5>(mode, a, rows, s, lazy);
        case 6: return launch_mode<6>(mode, a, rows, s, lazy);
        case 7: return launch_mode<7>(mode, a, rows, s, lazy);
        case 8: return launch_mode<8>(mode, a, rows, s, lazy);
        case 9: return launch_mode<9>(mode, a, rows, s, lazy);
        case 10: return launch_mode<10>(mode, a, rows, s, lazy);
        case 11: return launch_mode<11>(mode, a, rows, s, lazy);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cc
}  // namespace hefx
