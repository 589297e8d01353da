// Elementwise kernels of HE-Mult (App. A: HE operators are built from NTT, INTT, BConv,
// VecModMul and VecModAdd): VecModMul, VecModAdd, the ciphertext tensor product, the
// key-switching inner product and Rescale.  Both operands of a product are runtime
// residues, so BAT (which needs one known factor) does not apply; the product is two
// Montgomery REDCs: mont(mont(x, y), 2^64 mod q) = x y mod q.  All are HBM-bound
// (vectorized 16-byte accesses, grid sized to the SM count).
#include <algorithm>

#include "hefx_internal.h"
#include "modarith.cuh"

namespace hefx {
namespace {

__device__ __forceinline__ uint32_t mulmod(uint32_t x, uint32_t y, const LimbConst& c) {
    const uint32_t t = mul_mont_lazy(x, y, c.q, c.qinv_neg);  // x y 2^-32, [0, 2q)
    return csub(mul_mont_lazy(t, c.r2, c.q, c.qinv_neg), c.q);
}

// Barrett variant of the same product (the paper's reduction ablation, Sec. V-F): quotient of
// the 64-bit product from floor(2^64 / q), one conditional subtraction.
__device__ __forceinline__ uint32_t mulmod_barrett(uint32_t x, uint32_t y, const LimbConst& c) {
    const uint64_t z = (uint64_t)x * y;
    const uint64_t mu = ((uint64_t)c.bar_hi << 32) | c.bar_lo;
    return csub((uint32_t)(z - __umul64hi(z, mu) * c.q), c.q);
}

template <bool BARRETT>
__global__ void __launch_bounds__(256) vec_mod_mul_kernel(const LimbConst* __restrict__ lc, uint32_t L, uint32_t n,
                                                          size_t total4, const uint4* x, const uint4* y, uint4* z) {
    griddep_wait();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total4; i += (size_t)gridDim.x * blockDim.x) {
        const LimbConst c = lc[((i * 4) / n) % L];
        const uint4 a = x[i], b = y[i];
        if constexpr (BARRETT)
            z[i] = make_uint4(mulmod_barrett(a.x, b.x, c), mulmod_barrett(a.y, b.y, c), mulmod_barrett(a.z, b.z, c),
                              mulmod_barrett(a.w, b.w, c));
        else
            z[i] = make_uint4(mulmod(a.x, b.x, c), mulmod(a.y, b.y, c), mulmod(a.z, b.z, c), mulmod(a.w, b.w, c));
    }
}

// z0 = x o y0, z1 = x o y1 (one key-switching operand times both key halves: x read once).
__global__ void __launch_bounds__(256) vec_mod_mul2_kernel(const LimbConst* __restrict__ lc, uint32_t L, uint32_t n,
                                                           size_t total4, const uint4* x, const uint4* y0,
                                                           const uint4* y1, uint4* z0, uint4* z1) {
    griddep_wait();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total4; i += (size_t)gridDim.x * blockDim.x) {
        const LimbConst c = lc[((i * 4) / n) % L];
        const uint4 a = x[i], b0 = y0[i], b1 = y1[i];
        z0[i] = make_uint4(mulmod(a.x, b0.x, c), mulmod(a.y, b0.y, c), mulmod(a.z, b0.z, c), mulmod(a.w, b0.w, c));
        z1[i] = make_uint4(mulmod(a.x, b1.x, c), mulmod(a.y, b1.y, c), mulmod(a.z, b1.z, c), mulmod(a.w, b1.w, c));
    }
}

__device__ __forceinline__ uint32_t mac2(uint32_t a, uint32_t b, uint32_t c, uint32_t d, const LimbConst& k) {
    // (a b + c d) mod q with one final pair of reductions
    const uint32_t t = mul_mont_lazy(a, b, k.q, k.qinv_neg) + mul_mont_lazy(c, d, k.q, k.qinv_neg);  // < 4q
    return csub(mul_mont_lazy(t, k.r2, k.q, k.qinv_neg), k.q);
}

__global__ void __launch_bounds__(256) tensor_product_kernel(const LimbConst* __restrict__ lc, uint32_t L, uint32_t n,
                                                             size_t total4, const uint4* a0, const uint4* a1,
                                                             const uint4* b0, const uint4* b1, uint4* d0, uint4* d1,
                                                             uint4* d2) {
    griddep_wait();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total4; i += (size_t)gridDim.x * blockDim.x) {
        const LimbConst c = lc[((i * 4) / n) % L];
        const uint4 x0 = a0[i], x1 = a1[i], y0 = b0[i], y1 = b1[i];
        d0[i] = make_uint4(mulmod(x0.x, y0.x, c), mulmod(x0.y, y0.y, c), mulmod(x0.z, y0.z, c), mulmod(x0.w, y0.w, c));
        d1[i] = make_uint4(mac2(x0.x, y1.x, x1.x, y0.x, c), mac2(x0.y, y1.y, x1.y, y0.y, c),
                           mac2(x0.z, y1.z, x1.z, y0.z, c), mac2(x0.w, y1.w, x1.w, y0.w, c));
        if (d2)  // null: d2 not wanted (HE-Mult takes INTT(a1 o b1) straight from the inputs)
            d2[i] =
                make_uint4(mulmod(x1.x, y1.x, c), mulmod(x1.y, y1.y, c), mulmod(x1.z, y1.z, c), mulmod(x1.w, y1.w, c));
    }
}

__global__ void __launch_bounds__(256) vec_mod_add_kernel(const LimbConst* __restrict__ lc, uint32_t L, uint32_t n,
                                                          size_t total4, const uint4* x, const uint4* y, uint4* z) {
    griddep_wait();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total4; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t q = lc[((i * 4) / n) % L].q;
        const uint4 a = x[i], b = y[i];
        z[i] = make_uint4(csub(a.x + b.x, q), csub(a.y + b.y, q), csub(a.z + b.z, q), csub(a.w + b.w, q));
    }
}

// Key-switching inner product: out[b][k][l] = sum_j dig[b][j][l] o evk[j][k][l] mod q_l over
// the nl limbs of Q u P.  Each term is one REDC (x y 2^-32 in [0, 2q)); the running sum is kept
// in [0, 2q) and one REDC by 2^64 mod q at the end removes the 2^-32.
__device__ __forceinline__ uint32_t kip_term(uint32_t acc, uint32_t x, uint32_t y, const LimbConst& c) {
    return csub(acc + mul_mont_lazy(x, y, c.q, c.qinv_neg), 2 * c.q);
}
__device__ __forceinline__ uint32_t kip_final(uint32_t acc, const LimbConst& c) {
    return csub(mul_mont_lazy(acc, c.r2, c.q, c.qinv_neg), c.q);
}

__global__ void __launch_bounds__(256) key_inner_product_kernel(const LimbConst* __restrict__ lc, uint32_t nl,
                                                                uint32_t n, uint32_t dnum, size_t batch,
                                                                const uint4* dig, const uint4* evk, uint4* out) {
    griddep_wait();
    const size_t per_poly4 = (size_t)nl * n / 4;  // uint4 groups of one polynomial over Q u P
    const size_t total4 = batch * per_poly4;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total4; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / per_poly4, e = i % per_poly4;
        const LimbConst c = lc[(e * 4) / n];
        uint4 a0 = make_uint4(0, 0, 0, 0), a1 = make_uint4(0, 0, 0, 0);
        for (uint32_t j = 0; j < dnum; ++j) {
            const uint4 d = dig[(b * dnum + j) * per_poly4 + e];
            const uint4 k0 = evk[(size_t)(2 * j) * per_poly4 + e], k1 = evk[(size_t)(2 * j + 1) * per_poly4 + e];
            a0 = make_uint4(kip_term(a0.x, d.x, k0.x, c), kip_term(a0.y, d.y, k0.y, c), kip_term(a0.z, d.z, k0.z, c),
                            kip_term(a0.w, d.w, k0.w, c));
            a1 = make_uint4(kip_term(a1.x, d.x, k1.x, c), kip_term(a1.y, d.y, k1.y, c), kip_term(a1.z, d.z, k1.z, c),
                            kip_term(a1.w, d.w, k1.w, c));
        }
        out[(2 * b) * per_poly4 + e] = make_uint4(kip_final(a0.x, c), kip_final(a0.y, c), kip_final(a0.z, c),
                                                  kip_final(a0.w, c));
        out[(2 * b + 1) * per_poly4 + e] = make_uint4(kip_final(a1.x, c), kip_final(a1.y, c), kip_final(a1.z, c),
                                                      kip_final(a1.w, c));
    }
}

// Rescale by the parameter set's last prime: out[b][i] = (x[b][i] - [x[b][L-1]]_{q_i}) * q_{L-1}^-1
// mod q_i for i < L - 1 (coefficient form).  x_{L-1} < q_{L-1} < 2^30 is brought into [0, q_i)
// by a Shoup product with 1 and one subtraction.
__global__ void __launch_bounds__(256) rescale_kernel(const LimbConst* __restrict__ lc, uint32_t L, uint32_t n,
                                                      size_t batch, const uint4* x, uint4* out) {
    griddep_wait();
    const size_t row4 = n / 4;
    const size_t per_out4 = (size_t)(L - 1) * row4;
    const size_t total4 = batch * per_out4;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total4; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / per_out4, e = i % per_out4;
        const size_t limb = e / row4, col = e % row4;
        const LimbConst c = lc[limb];
        const uint4 v = x[(b * L + limb) * row4 + col], t = x[(b * L + L - 1) * row4 + col];
        auto one = [&](uint32_t xv, uint32_t tv) {
            const uint32_t last = csub(mul_shoup_lazy(tv, 1u, c.one_sh, c.q), c.q);
            return csub(mul_shoup_lazy(xv + c.q - last, c.rs_inv, c.rs_inv_sh, c.q), c.q);
        };
        out[i] = make_uint4(one(v.x, t.x), one(v.y, t.y), one(v.z, t.z), one(v.w, t.w));
    }
}

unsigned grid_for(size_t total4) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (unsigned)std::max<size_t>(1, std::min<size_t>((total4 + 255) / 256, (size_t)sms * 8));
}

}  // namespace

cudaError_t launch_vec_mod_mul(const hefx_params* p, const uint32_t* x, const uint32_t* y, uint32_t* z, size_t rows,
                               cudaStream_t s) {
    const size_t total4 = rows * p->n / 4;  // N >= 8, so rows of N words split into whole uint4
    if (!total4) return cudaSuccess;
    if (p->red_vec == HEFX_RED_BAT_LAZY) return launch_vec_mod_mul_bat(p, x, y, z, rows, s);
    if (p->red_vec == HEFX_RED_BARRETT)
        return launch_pdl(vec_mod_mul_kernel<true>, grid_for(total4), 256, 0, s, (const LimbConst*)p->d_lc, p->nlimbs,
                          p->n, total4, (const uint4*)x, (const uint4*)y, (uint4*)z);
    else
        return launch_pdl(vec_mod_mul_kernel<false>, grid_for(total4), 256, 0, s, (const LimbConst*)p->d_lc, p->nlimbs,
                          p->n, total4, (const uint4*)x, (const uint4*)y, (uint4*)z);
}

cudaError_t launch_vec_mod_mul2(const hefx_params* p, const uint32_t* x, const uint32_t* y0, const uint32_t* y1,
                                uint32_t* z0, uint32_t* z1, size_t rows, cudaStream_t s) {
    const size_t total4 = rows * p->n / 4;
    if (!total4) return cudaSuccess;
    if (p->red_vec != HEFX_RED_MONTGOMERY) {  // the other reductions: two single products
        cudaError_t e = launch_vec_mod_mul(p, x, y0, z0, rows, s);
        return e == cudaSuccess ? launch_vec_mod_mul(p, x, y1, z1, rows, s) : e;
    }
    return launch_pdl(vec_mod_mul2_kernel, grid_for(total4), 256, 0, s, (const LimbConst*)p->d_lc, p->nlimbs, p->n,
                      total4, (const uint4*)x, (const uint4*)y0, (const uint4*)y1, (uint4*)z0, (uint4*)z1);
}

cudaError_t launch_tensor_product(const hefx_params* p, const uint32_t* a0, const uint32_t* a1, const uint32_t* b0,
                                  const uint32_t* b1, uint32_t* d0, uint32_t* d1, uint32_t* d2, size_t rows,
                                  cudaStream_t s) {
    const size_t total4 = rows * p->n / 4;
    if (!total4) return cudaSuccess;
    return launch_pdl(tensor_product_kernel, grid_for(total4), 256, 0, s, (const LimbConst*)p->d_lc, p->nlimbs, p->n,
                      total4, (const uint4*)a0, (const uint4*)a1, (const uint4*)b0, (const uint4*)b1, (uint4*)d0,
                      (uint4*)d1, (uint4*)d2);
}

cudaError_t launch_vec_mod_add(const hefx_params* p, const uint32_t* x, const uint32_t* y, uint32_t* z, size_t rows,
                               cudaStream_t s) {
    const size_t total4 = rows * p->n / 4;
    if (!total4) return cudaSuccess;
    return launch_pdl(vec_mod_add_kernel, grid_for(total4), 256, 0, s, (const LimbConst*)p->d_lc, p->nlimbs, p->n,
                      total4, (const uint4*)x, (const uint4*)y, (uint4*)z);
}

cudaError_t launch_key_inner_product(const hefx_params* p, const uint32_t* dig, const uint32_t* evk, uint32_t* out,
                                     uint32_t dnum, size_t batch, cudaStream_t s) {
    const size_t total4 = batch * p->nlimbs * p->n / 4;
    if (!total4) return cudaSuccess;
    return launch_pdl(key_inner_product_kernel, grid_for(total4), 256, 0, s, (const LimbConst*)p->d_lc, p->nlimbs, p->n,
                      dnum, batch, (const uint4*)dig, (const uint4*)evk, (uint4*)out);
}

cudaError_t launch_rescale(const hefx_params* p, const uint32_t* x, uint32_t* out, size_t batch, cudaStream_t s) {
    const size_t total4 = batch * (p->nlimbs - 1) * p->n / 4;
    if (!total4) return cudaSuccess;
    return launch_pdl(rescale_kernel, grid_for(total4), 256, 0, s, (const LimbConst*)p->d_lc, p->nlimbs, p->n, batch,
                      (const uint4*)x, (uint4*)out);
}

}  // namespace hefx
