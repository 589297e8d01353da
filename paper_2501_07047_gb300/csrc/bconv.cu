// RNS basis conversion (App. B, BConv), CUDA-core path and plan constants.
//
//   out_{n,j} = sum_i [a_{n,i} * qhat_i^-1]_{q_i} * [qhat_i]_{p_j}  mod p_j
//
// The same kernel with a ModDown epilogue finishes hybrid key switching (the HE-Mult of
// Sec. V-A): with the plan's sources the special primes P and its targets the ciphertext
// primes, out_{n,j} = (x_{n,j} - BConv(x_P)_{n,j}) * P^-1 mod q_j.  Its exact variant
// subtracts v Q with v = round(sum_i b_i / q_i), estimated as a 128-bit fixed-point sum
// sum_i b_i round(2^k / q_i) (error below 2^-55 Q), which yields the centered CRT value
// mod p_j (the u-corrected conversion; the paper prints only the fast one).
//
// Step 1 is L independent VecModMuls by the constant qhat_i^-1 (Shoup products); step 2
// is an (N, L, L') MatModMul whose right operand is the constant matrix [qhat_i]_{p_j}.
// This file runs step 2 as 64-bit multiply-accumulates (each product < 2^58, L <= 64
// products fit in 64 bits) with one Barrett reduction per output; bconv_tc.cu runs it on
// the tensor cores as a digit-split (BAT) matrix product.
#include <algorithm>

#include "bconv_common.h"
#include "host_nt.h"
#include "modarith.cuh"

namespace hefx {

cudaError_t bconv_plan_upload(hefx_bconv_plan* plan) {
    const uint32_t L = plan->L, Lp = plan->Lp;
    BConvConst h;
    memset(&h, 0, sizeof(h));
    h.L = L;
    h.Lp = Lp;
    for (uint32_t i = 0; i < L; ++i) {
        const uint64_t q = plan->src[i];
        uint64_t qhat = 1;
        for (uint32_t k = 0; k < L; ++k)
            if (k != i) qhat = mul_mod(qhat, plan->src[k], q);
        const uint64_t qi = inv_mod(qhat, q);
        h.q[i] = (uint32_t)q;
        h.qhat_inv[i] = (uint32_t)qi;
        h.qhat_inv_sh[i] = shoup(qi, q);
        for (uint32_t j = 0; j < Lp; ++j) {
            uint64_t c = 1;
            for (uint32_t k = 0; k < L; ++k)
                if (k != i) c = mul_mod(c, plan->src[k], plan->dst[j]);
            h.qhat_p[i * kBConvMaxLimbs + j] = (uint32_t)c;
        }
    }
    for (uint32_t j = 0; j < Lp; ++j) {
        h.p[j] = plan->dst[j];
        h.p_mu[j] = (uint64_t)(((u128)1 << 64) / plan->dst[j]);  // floor(2^64 / p_j)
        uint64_t prod = 1;
        for (uint32_t i = 0; i < L; ++i) prod = mul_mod(prod, plan->src[i], plan->dst[j]);
        const uint64_t pinv = inv_mod(prod, plan->dst[j]);
        h.pinv[j] = (uint32_t)pinv;
        h.pinv_sh[j] = shoup(pinv, plan->dst[j]);
        h.qmod_p[j] = (uint32_t)prod;
    }
    // exact conversion: k = 63 + floor(log2(min q_i)) keeps every w_i = round(2^k / q_i) below 2^64
    uint32_t minq = plan->src[0];
    for (uint32_t i = 1; i < L; ++i) minq = std::min(minq, plan->src[i]);
    int lg = 0;
    while ((2u << lg) <= minq) ++lg;
    const int k = 63 + lg;
    for (uint32_t i = 0; i < L; ++i) {
        const u128 num = (u128)1 << k;
        const u128 qi = plan->src[i];
        h.w[i] = (uint64_t)((num + qi / 2) / qi);
    }
    const u128 half = (u128)1 << (k - 1);
    h.half_lo = (uint64_t)half;
    h.half_hi = (uint64_t)(half >> 64);
    h.kshift = (uint32_t)(k - 64);
    cudaError_t e = cudaMalloc(&plan->d_const, sizeof(BConvConst));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(plan->d_const, &h, sizeof(BConvConst), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    return bconv_tc_upload(plan, h);
}

void bconv_plan_free(hefx_bconv_plan* plan) {
    if (plan->d_const) cudaFree(plan->d_const);
    plan->d_const = nullptr;
    bconv_tc_free(plan);
}

namespace {

constexpr int kJChunk = 8;  // target limbs accumulated per pass over the source limbs

__device__ __forceinline__ uint32_t barrett64(uint64_t x, uint32_t p, uint64_t mu) {
    const uint64_t qt = __umul64hi(x, mu);  // floor(x / p) or one less
    uint64_t r = x - qt * p;
    return (uint32_t)(r >= p ? r - p : r);
}

// kCoef coefficients per thread: each constant load serves kCoef products (1 for n < 4).
// Polynomial b's source limbs start at in + b * in_stride, its outputs at out + b * out_stride.
// MODE 1 (ModDown): the epilogue returns (x_j - conv_j) * P^-1 mod p_j, x_j at
// xq + b * in_stride + j n.  MODE 2 (exact): conv_j - v [Q]_{p_j}, v = round(sum_i b_i / q_i).
enum : int { BC_FAST = 0, BC_MODDOWN = 1, BC_EXACT = 2 };

template <int kCoef, int MODE>
__global__ void __launch_bounds__(256) bconv_cc_kernel(const BConvConst* __restrict__ gc, const uint32_t* __restrict__ in,
                                                       uint32_t* __restrict__ out, const uint32_t* __restrict__ xq,
                                                       uint32_t n, uint32_t batch, size_t in_stride,
                                                       size_t out_stride) {
    __shared__ BConvConst c;
    for (int i = threadIdx.x; i < (int)(sizeof(BConvConst) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(&c)[i] = reinterpret_cast<const uint32_t*>(gc)[i];
    __syncthreads();
    const uint32_t L = c.L, Lp = c.Lp;
    const size_t groups = (size_t)n * batch / kCoef;  // n is a multiple of kCoef
    // one thread per (group of kCoef coefficients, chunk of kJChunk target limbs): the chunk is
    // the slow index, so the lanes of a warp read consecutive coefficients
    const uint32_t nchunks = (Lp + kJChunk - 1) / kJChunk;
    for (size_t tt = blockIdx.x * (size_t)blockDim.x + threadIdx.x; tt < groups * nchunks;
         tt += (size_t)gridDim.x * blockDim.x) {
        const size_t t = tt % groups;
        const uint32_t j0 = (uint32_t)(tt / groups) * kJChunk;
        // kCoef coefficients x, x + stride, ... of one polynomial (stride keeps warps coalesced)
        const size_t per_poly = n / kCoef;
        const size_t b = t / per_poly, x0 = t % per_poly;
        const uint32_t* src = in + b * in_stride + x0;
        uint32_t* dst = out + b * out_stride + x0;
        uint32_t v[kCoef];  // exact conversion: the multiple of Q to remove
        if constexpr (MODE == BC_EXACT) {
#pragma unroll
            for (int u = 0; u < kCoef; ++u) {
                uint64_t lo = c.half_lo, hi = c.half_hi;
                for (uint32_t i = 0; i < L; ++i) {
                    const uint32_t qi = c.q[i];
                    const uint32_t bi = csub(mul_shoup_lazy(__ldg(src + (size_t)i * n + u * per_poly), c.qhat_inv[i],
                                                            c.qhat_inv_sh[i], qi), qi);
                    const uint64_t plo = (uint64_t)bi * c.w[i], phi = __umul64hi((uint64_t)bi, c.w[i]);
                    lo += plo;
                    hi += phi + (lo < plo ? 1u : 0u);
                }
                v[u] = (uint32_t)(hi >> c.kshift);
            }
        }
        {
            uint64_t acc[kCoef][kJChunk];
#pragma unroll
            for (int u = 0; u < kCoef; ++u)
#pragma unroll
                for (int jj = 0; jj < kJChunk; ++jj) acc[u][jj] = 0;
            for (uint32_t i = 0; i < L; ++i) {
                uint32_t v[kCoef];
#pragma unroll
                for (int u = 0; u < kCoef; ++u) v[u] = __ldg(src + (size_t)i * n + u * per_poly);
                const uint32_t qi = c.q[i], w = c.qhat_inv[i], wsh = c.qhat_inv_sh[i];
                uint32_t cst[kJChunk];
#pragma unroll
                for (int jj = 0; jj < kJChunk; ++jj) cst[jj] = c.qhat_p[i * kBConvMaxLimbs + j0 + jj];
#pragma unroll
                for (int u = 0; u < kCoef; ++u) {
                    const uint32_t bi = csub(mul_shoup_lazy(v[u], w, wsh, qi), qi);  // step 1
#pragma unroll
                    for (int jj = 0; jj < kJChunk; ++jj) acc[u][jj] += (uint64_t)bi * cst[jj];  // step 2
                }
            }
#pragma unroll
            for (int jj = 0; jj < kJChunk; ++jj) {
                const uint32_t j = j0 + jj;
                if (j < Lp) {
#pragma unroll
                    for (int u = 0; u < kCoef; ++u) {
                        uint32_t r = barrett64(acc[u][jj], c.p[j], c.p_mu[j]);
                        if constexpr (MODE == BC_EXACT) {
                            const uint32_t corr = barrett64((uint64_t)v[u] * c.qmod_p[j], c.p[j], c.p_mu[j]);
                            r = csub(r + c.p[j] - corr, c.p[j]);
                        }
                        if constexpr (MODE == BC_MODDOWN) {
                            const uint32_t pj = c.p[j];
                            const uint32_t x = __ldg(xq + b * in_stride + (size_t)j * n + x0 + u * per_poly);
                            r = csub(mul_shoup_lazy(x + pj - r, c.pinv[j], c.pinv_sh[j], pj), pj);
                        }
                        dst[(size_t)j * n + u * per_poly] = r;
                    }
                }
            }
        }
    }
}

unsigned bconv_blocks(size_t total, uint32_t Lp) {
    total *= (Lp + kJChunk - 1) / kJChunk;
    size_t blocks = (total + 255) / 256;  // one (coefficient, target chunk) per thread, many short blocks
    const size_t cap = (size_t)1 << 20;
    return (unsigned)(blocks > cap ? cap : blocks);
}

}  // namespace

cudaError_t launch_bconv_cc(const hefx_bconv_plan* plan, const uint32_t* in, uint32_t* out, size_t batch,
                            cudaStream_t stream) {
    const uint32_t n = 1u << plan->log2n;
    const size_t total = (size_t)n * batch;
    if (total == 0) return cudaSuccess;
    // measured: 4 coefficients per thread (95 registers) is slower than 1
    bconv_cc_kernel<1, BC_FAST><<<bconv_blocks(total, plan->Lp), 256, 0, stream>>>(
        static_cast<const BConvConst*>(plan->d_const), in, out, nullptr, n, (uint32_t)batch, (size_t)plan->L * n,
        (size_t)plan->Lp * n);
    return cudaGetLastError();
}

cudaError_t launch_bconv_exact(const hefx_bconv_plan* plan, const uint32_t* in, uint32_t* out, size_t batch,
                               cudaStream_t stream) {
    const uint32_t n = 1u << plan->log2n;
    const size_t total = (size_t)n * batch;
    if (total == 0) return cudaSuccess;
    bconv_cc_kernel<1, BC_EXACT><<<bconv_blocks(total, plan->Lp), 256, 0, stream>>>(
        static_cast<const BConvConst*>(plan->d_const), in, out, nullptr, n, (uint32_t)batch, (size_t)plan->L * n,
        (size_t)plan->Lp * n);
    return cudaGetLastError();
}

cudaError_t launch_mod_down(const hefx_bconv_plan* plan, const uint32_t* x, uint32_t* out, size_t batch,
                            cudaStream_t stream) {
    // x: [batch][Lp + L][n] (target-basis limbs first, then the plan's source limbs)
    const uint32_t n = 1u << plan->log2n;
    const size_t total = (size_t)n * batch;
    if (total == 0) return cudaSuccess;
    const size_t stride = (size_t)(plan->L + plan->Lp) * n;
    bconv_cc_kernel<1, BC_MODDOWN><<<bconv_blocks(total, plan->Lp), 256, 0, stream>>>(
        static_cast<const BConvConst*>(plan->d_const), x + (size_t)plan->Lp * n, out, x, n, (uint32_t)batch, stride,
        (size_t)plan->Lp * n);
    return cudaGetLastError();
}

}  // namespace hefx
