// Basis-conversion plan constants shared by the CUDA-core and tensor-core BConv kernels.
#pragma once

#include <cstddef>
#include <cstring>

#include "hefx_internal.h"

namespace hefx {

constexpr int kBConvMaxLimbs = 64;

struct BConvConst {
    uint32_t L, Lp;
    uint32_t skip_lo, skip_len;            // ModUp: target j is written at row j + (j >= skip_lo ? skip_len : 0)
    uint32_t q[kBConvMaxLimbs];            // source primes q_i
    uint32_t qhat_inv[kBConvMaxLimbs];     // qhat_i^-1 mod q_i (step 1 constant)
    uint32_t qhat_inv_sh[kBConvMaxLimbs];  // its Shoup companion
    uint32_t p[kBConvMaxLimbs];            // target primes p_j
    uint64_t p_mu[kBConvMaxLimbs];         // floor(2^64 / p_j) (Barrett)
    uint32_t pinv[kBConvMaxLimbs];         // (prod_i q_i)^-1 mod p_j (ModDown scale)
    uint32_t pinv_sh[kBConvMaxLimbs];      // its Shoup companion
    uint32_t qmod_p[kBConvMaxLimbs];       // Q mod p_j (exact conversion's correction)
    uint64_t w[kBConvMaxLimbs];            // round(2^k / q_i) (exact conversion's estimate of u)
    uint64_t half_lo, half_hi;             // 2^(k-1) as a 128-bit value
    uint32_t kshift, pad2, pad3[2];        // k - 64
    uint32_t qpack[kBConvMaxLimbs][4];     // (q_i, qhat_i^-1, its Shoup companion, 0): one 16-byte load
    uint32_t qhat_p[kBConvMaxLimbs * kBConvMaxLimbs];  // [i][j] = qhat_i mod p_j (step 2 matrix)
};
// 16-byte aligned rows: the kernels read the matrix and copy the struct as uint4
static_assert(offsetof(BConvConst, qhat_p) % 16 == 0 && sizeof(BConvConst) % 16 == 0, "BConvConst layout");

// x mod p for a 64-bit x, with mu = floor(2^64 / p) (Barrett): the estimated quotient is
// floor(x / p) or one less, so one conditional subtraction finishes.
__device__ __forceinline__ uint32_t barrett64(uint64_t x, uint32_t p, uint64_t mu) {
    const uint64_t qt = __umul64hi(x, mu);
    const uint64_t r = x - qt * p;
    return (uint32_t)(r >= p ? r - p : r);
}

// Host: the plan constants of a conversion from src[0..L) to dst[0..Lp) (skip fields 0).
void fill_bconv_const(const uint32_t* src, uint32_t L, const uint32_t* dst, uint32_t Lp, BConvConst& h);

cudaError_t bconv_tc_upload(hefx_bconv_plan* plan, const BConvConst& h);
void bconv_tc_free(hefx_bconv_plan* plan);
bool bconv_tc_available(const hefx_bconv_plan* plan);
// The path HEFX_PATH_AUTO takes for a call of `batch` polynomials (measured rule: the tensor
// path wins only with more than 8 targets on throughput-sized calls).
bool bconv_prefer_tc(const hefx_bconv_plan* plan, size_t batch);

}  // namespace hefx
