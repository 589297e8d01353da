// Elementwise modular products of the HE-Mult request: VecModMul and the ciphertext tensor
// product (Sec. III: HE-Mult = tensor product, then key switching built from INTT, BConv,
// NTT and VecModMul).  Both operands are runtime residues, so BAT (which needs one known
// factor) does not apply; the product is two Montgomery REDCs: mont(mont(x, y), 2^64 mod q)
// = x y mod q.  HBM-bound: 12 bytes (VecModMul) or 28 bytes (tensor product) per
// coefficient, vectorized 16-byte accesses, grid sized to the SM count.
#include <algorithm>

#include "hefx_internal.h"
#include "modarith.cuh"

namespace hefx {
namespace {

__device__ __forceinline__ uint32_t mulmod(uint32_t x, uint32_t y, const LimbConst& c) {
    const uint32_t t = mul_mont_lazy(x, y, c.q, c.qinv_neg);  // x y 2^-32, [0, 2q)
    return csub(mul_mont_lazy(t, c.r2, c.q, c.qinv_neg), c.q);
}

__global__ void __launch_bounds__(256) vec_mod_mul_kernel(const LimbConst* __restrict__ lc, uint32_t L, uint32_t n,
                                                          size_t total4, const uint4* x, const uint4* y, uint4* z) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total4; i += (size_t)gridDim.x * blockDim.x) {
        const LimbConst c = lc[((i * 4) / n) % L];
        const uint4 a = x[i], b = y[i];
        z[i] = make_uint4(mulmod(a.x, b.x, c), mulmod(a.y, b.y, c), mulmod(a.z, b.z, c), mulmod(a.w, b.w, c));
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
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total4; i += (size_t)gridDim.x * blockDim.x) {
        const LimbConst c = lc[((i * 4) / n) % L];
        const uint4 x0 = a0[i], x1 = a1[i], y0 = b0[i], y1 = b1[i];
        d0[i] = make_uint4(mulmod(x0.x, y0.x, c), mulmod(x0.y, y0.y, c), mulmod(x0.z, y0.z, c), mulmod(x0.w, y0.w, c));
        d1[i] = make_uint4(mac2(x0.x, y1.x, x1.x, y0.x, c), mac2(x0.y, y1.y, x1.y, y0.y, c),
                           mac2(x0.z, y1.z, x1.z, y0.z, c), mac2(x0.w, y1.w, x1.w, y0.w, c));
        d2[i] = make_uint4(mulmod(x1.x, y1.x, c), mulmod(x1.y, y1.y, c), mulmod(x1.z, y1.z, c), mulmod(x1.w, y1.w, c));
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
    vec_mod_mul_kernel<<<grid_for(total4), 256, 0, s>>>(p->d_lc, p->nlimbs, p->n, total4, (const uint4*)x,
                                                        (const uint4*)y, (uint4*)z);
    return cudaGetLastError();
}

cudaError_t launch_tensor_product(const hefx_params* p, const uint32_t* a0, const uint32_t* a1, const uint32_t* b0,
                                  const uint32_t* b1, uint32_t* d0, uint32_t* d1, uint32_t* d2, size_t rows,
                                  cudaStream_t s) {
    const size_t total4 = rows * p->n / 4;
    if (!total4) return cudaSuccess;
    tensor_product_kernel<<<grid_for(total4), 256, 0, s>>>(p->d_lc, p->nlimbs, p->n, total4, (const uint4*)a0,
                                                           (const uint4*)a1, (const uint4*)b0, (const uint4*)b1,
                                                           (uint4*)d0, (uint4*)d1, (uint4*)d2);
    return cudaGetLastError();
}

}  // namespace hefx
