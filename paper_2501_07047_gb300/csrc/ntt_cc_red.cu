// The N = 2^16 CUDA-core forward and inverse transforms with Montgomery and Barrett twiddle
// products: the variants of the paper's modular-reduction ablation (Sec. V-F, "Impact of
// Modular Reduction Algorithm").  Shoup products, the default, live in ntt_cc_range_d.cu.
#include <cstring>

#include "ntt_cc_impl.cuh"

namespace hefx {
namespace cc {
namespace {

template <int F>
cudaError_t red_launch(NttMode mode, const KArgs& a, size_t rows, cudaStream_t s) {
    switch (mode) {
        case MODE_FWD: return launch_one<16, MODE_FWD, F>(a, rows, s);
        case MODE_INV: return launch_one<16, MODE_INV, F>(a, rows, s);
        default: return cudaErrorNotSupported;
    }
}

// Montgomery form of a twiddle table: w -> w 2^32 mod q, as REDC(w * (2^64 mod q)).
__global__ void __launch_bounds__(256) mont_table_kernel(const LimbConst* __restrict__ lc, uint32_t n, size_t total,
                                                          const uint2* __restrict__ tw, uint2* __restrict__ out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const LimbConst& c = lc[i / n];
        out[i] = make_uint2(csub(mul_mont_lazy(tw[i].x, c.r2, c.q, c.qinv_neg), c.q), 0u);
    }
}

}  // namespace
}  // namespace cc

cudaError_t launch_ntt_cc_red(const hefx_params* p, NttMode mode, uint32_t* data, size_t rows, cudaStream_t stream) {
    if (p->log2n != 16 || (mode != MODE_FWD && mode != MODE_INV)) return cudaErrorNotSupported;
    if (rows == 0) return cudaSuccess;
    cc::KArgs a;
    memset(&a.tmap_in, 0, sizeof a.tmap_in);
    memset(&a.tmap_out, 0, sizeof a.tmap_out);
    a.err = p->d_err_cc;
    cudaError_t em = encode_input_map(p, data, rows, mode == MODE_INV ? &a.tmap_in : &a.tmap_out);
    if (em != cudaSuccess) return em;
    a.in = data;
    a.had = nullptr;
    a.out = data;
    a.tw_f = p->red_ntt == HEFX_RED_MONTGOMERY ? p->d_tw_fwd_mont : p->d_tw_fwd;
    a.tw_i = p->red_ntt == HEFX_RED_MONTGOMERY ? p->d_tw_inv_mont : p->d_tw_inv;
    if (!a.tw_f || !a.tw_i) return cudaErrorNotSupported;
    a.lc = p->d_lc;
    a.desc = nullptr;
    a.in_rows = 0;
    a.rows = (uint32_t)rows;
    a.L = p->nlimbs;
    const bool lazy = p->max_prime < (1u << 28);
    if (p->red_ntt == HEFX_RED_MONTGOMERY)
        return lazy ? cc::red_launch<2 | (1 << 2)>(mode, a, rows, stream) : cc::red_launch<1 << 2>(mode, a, rows, stream);
    if (p->red_ntt == HEFX_RED_BARRETT)
        return lazy ? cc::red_launch<2 | (2 << 2)>(mode, a, rows, stream) : cc::red_launch<2 << 2>(mode, a, rows, stream);
    return cudaErrorNotSupported;
}

cudaError_t make_mont_twiddles(const hefx_params* p, const uint2* tw, uint2* out) {
    const size_t total = (size_t)p->nlimbs * p->n;
    cc::mont_table_kernel<<<(unsigned)std::min<size_t>((total + 255) / 256, 4096), 256>>>(p->d_lc, p->n, total, tw, out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e;
}

}  // namespace hefx
