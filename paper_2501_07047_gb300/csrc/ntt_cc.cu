// CUDA-core NTT dispatcher and public launchers; the kernels are in ntt_cc_impl.cuh and are
// instantiated per ring-degree range in ntt_cc_range_*.cu (parallel compilation).
#include <cstring>

#include "ntt_cc_impl.cuh"

namespace hefx {

cudaError_t launch_dispatch(const hefx_params* p, NttMode mode, const cc::KArgs& a, size_t rows, cudaStream_t stream);

namespace {

// Co-resident clusters of the N = 2^16 forward / inverse kernel, queried once per context.
int clusters16(hefx_ctx* c, NttMode mode, bool lazy) {
    std::lock_guard<std::mutex> g(c->mu);
    int& v = c->cc16_clusters[mode == MODE_INV ? 1 : 0][lazy ? 1 : 0];
    if (v < 0) v = cc::max_clusters_16(mode, lazy);
    return v;
}

}  // namespace

// Tensor map of a contiguous [rows][N] input for the inverse transforms' TMA loads.
cudaError_t encode_input_map(const hefx_params* p, const uint32_t* in, size_t rows, CUtensorMap* map) {
    const uint64_t lines = (uint64_t)rows * p->n / 32;  // 128-byte lines of 32 words
    if (!encode_map_2d(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, const_cast<uint32_t*>(in), 32, lines, 128, 32, 256,
                       CU_TENSOR_MAP_SWIZZLE_128B))
        return cudaErrorNotSupported;
    return cudaSuccess;
}

cudaError_t launch_ntt_cc(const hefx_params* p, NttMode mode, const uint32_t* in, const uint32_t* had, uint32_t* out,
                          size_t rows, cudaStream_t stream) {
    // AUTO takes the two-pass schedule where it measured faster than the clusters: up to 32
    // rows (one polynomial of 24 limbs: 16.7 / 16.4 us against 20.7 / 20.5 us), and from one
    // to one and a half waves of co-resident clusters, where the cluster kernel's second wave
    // is mostly empty (96 rows: 34.1 / 31.7 us against 35.6 / 34.8 us; 120 rows: 43.3 / 39.9
    // against 45.6 / 45.1 us); elsewhere the two are within a few percent and the single
    // launch stays
    bool two_pass = p->cc_schedule == HEFX_CC_TWO_PASS;
    if (p->cc_schedule == HEFX_CC_AUTO && ntt_cc_2p_supported(p, mode)) {
        constexpr size_t kTwoPassAutoRows = 32;
        if (rows <= kTwoPassAutoRows) {
            two_pass = true;
        } else {
            const size_t slots = (size_t)clusters16(p->ctx, mode, p->max_prime < (1u << 28));
            two_pass = slots > 0 && rows > slots && 2 * rows <= 3 * slots;
        }
    }
    if (two_pass && ntt_cc_2p_supported(p, mode)) return launch_ntt_cc_2p(p, mode, in, out, rows, stream);
    cc::KArgs a;
    memset(&a.tmap_in, 0, sizeof a.tmap_in);
    memset(&a.tmap_out, 0, sizeof a.tmap_out);
    a.err = p->d_err_cc;
    if (mode == MODE_INV && rows > 0 && p->log2n >= 13) {
        cudaError_t e = encode_input_map(p, in, rows, &a.tmap_in);
        if (e != cudaSuccess) return e;
    }
    if (mode == MODE_FWD && rows > 0 && p->log2n >= 13) {
        cudaError_t e = encode_input_map(p, out, rows, &a.tmap_out);
        if (e != cudaSuccess) return e;
    }
    a.in = in;
    a.had = had;
    a.out = out;
    a.tw_f = p->d_tw_fwd;
    a.tw_i = p->d_tw_inv;
    a.lc = p->d_lc;
    a.desc = nullptr;
    a.rows = (uint32_t)rows;
    a.L = p->nlimbs;
    a.in_rows = 0;
    if (rows == 0) return cudaSuccess;
    return launch_dispatch(p, mode, a, rows, stream);
}

cudaError_t launch_ntt_cc_rescale(const hefx_params* p, const uint32_t* in, uint32_t* out, size_t batch,
                                  cudaStream_t stream) {
    const uint32_t L = p->nlimbs;
    const size_t rows = batch * (L - 1);
    if (rows == 0) return cudaSuccess;
    cc::KArgs a;
    memset(&a.tmap_in, 0, sizeof a.tmap_in);
    memset(&a.tmap_out, 0, sizeof a.tmap_out);
    a.err = p->d_err_cc;
    if (p->log2n >= 13) {
        cudaError_t e = encode_input_map(p, out, rows, &a.tmap_out);
        if (e != cudaSuccess) return e;
    }
    a.in = in;
    a.had = nullptr;
    a.out = out;
    a.tw_f = p->d_tw_fwd;  // limbs 0 .. L-2 of the full set: the tables of q_0 .. q_{L-2}
    a.tw_i = p->d_tw_inv;
    a.lc = p->d_lc;        // rs_inv: q_{L-1}^-1 mod q_i
    a.desc = nullptr;
    a.rows = (uint32_t)rows;
    a.L = L - 1;
    a.in_rows = L;
    cudaError_t e = launch_dispatch(p, MODE_RS_FWD, a, rows, stream);
    if (e != cudaErrorNotSupported) return e;
    // not fused at this N: rescale into out, then the forward transform of its L - 1 limbs
    e = launch_rescale(p, in, out, batch, stream);
    if (e != cudaSuccess) return e;
    a.in = out;
    a.in_rows = 0;
    return launch_dispatch(p, MODE_FWD, a, rows, stream);
}

cudaError_t prepare_ntt_cc(const hefx_params* p, NttMode mode) {
    static const RowDesc dummy = {};
    cc::KArgs a = {};
    a.err = p->d_err_cc;
    a.desc = &dummy;  // selects the row-list kernels; rows == 0 sets attributes without launching
    return launch_dispatch(p, mode, a, 0, nullptr);
}

cudaError_t launch_ntt_cc_rows(const hefx_params* p, NttMode mode, const RowDesc* d_rows, size_t nrows,
                               cudaStream_t stream) {
    cc::KArgs a;
    memset(&a.tmap_in, 0, sizeof a.tmap_in);
    memset(&a.tmap_out, 0, sizeof a.tmap_out);
    a.err = p->d_err_cc;
    a.in = nullptr;
    a.had = nullptr;
    a.out = nullptr;
    a.tw_f = p->d_tw_fwd;
    a.tw_i = p->d_tw_inv;
    a.lc = p->d_lc;
    a.desc = d_rows;
    a.rows = (uint32_t)nrows;
    a.L = p->nlimbs;
    a.in_rows = 0;
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
