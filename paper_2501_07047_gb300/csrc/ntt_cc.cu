// CUDA-core NTT dispatcher and public launchers; the kernels are in ntt_cc_impl.cuh and are
// instantiated per ring-degree range in ntt_cc_range_*.cu (parallel compilation).
#include "ntt_cc_impl.cuh"

namespace hefx {

cudaError_t launch_dispatch(const hefx_params* p, NttMode mode, const cc::KArgs& a, size_t rows, cudaStream_t stream);

cudaError_t launch_ntt_cc(const hefx_params* p, NttMode mode, const uint32_t* in, const uint32_t* had, uint32_t* out,
                          size_t rows, cudaStream_t stream) {
    cc::KArgs a;
    a.in = in;
    a.had = had;
    a.out = out;
    a.tw_f = p->d_tw_fwd;
    a.tw_i = p->d_tw_inv;
    a.lc = p->d_lc;
    a.desc = nullptr;
    a.rows = (uint32_t)rows;
    a.L = p->nlimbs;
    if (rows == 0) return cudaSuccess;
    return launch_dispatch(p, mode, a, rows, stream);
}

cudaError_t prepare_ntt_cc(const hefx_params* p, NttMode mode) {
    static const RowDesc dummy = {};
    cc::KArgs a = {};
    a.desc = &dummy;  // selects the row-list kernels; rows == 0 sets attributes without launching
    return launch_dispatch(p, mode, a, 0, nullptr);
}

cudaError_t launch_ntt_cc_rows(const hefx_params* p, NttMode mode, const RowDesc* d_rows, size_t nrows,
                               cudaStream_t stream) {
    cc::KArgs a;
    a.in = nullptr;
    a.had = nullptr;
    a.out = nullptr;
    a.tw_f = p->d_tw_fwd;
    a.tw_i = p->d_tw_inv;
    a.lc = p->d_lc;
    a.desc = d_rows;
    a.rows = (uint32_t)nrows;
    a.L = p->nlimbs;
    if (nrows == 0) return cudaSuccess;
    return launch_dispatch(p, mode, a, nrows, stream);
}

cudaError_t launch_dispatch(const hefx_params* p, NttMode mode, const cc::KArgs& a, size_t rows, cudaStream_t stream) {
    const bool lazy = p->max_prime < (1u << 28);
    const int L = (int)p->log2n;
    if (L >= 3 && L <= 11) return cc::launch_range_a(L, mode, a, rows, stream, lazy);
    if (L >= 12 && L <= 14) return cc::launch_range_b(L, mode, a, rows, stream, lazy);
    if (L == 15) return cc::launch_range_c(L, mode, a, rows, stream, lazy);
    if (L == 16) return cc::launch_range_d(L, mode, a, rows, stream, lazy);
    if (L == 17) return cc::launch_range_e(L, mode, a, rows, stream, lazy);
    return cudaErrorInvalidValue;
}

}  // namespace hefx
