// Device modular arithmetic for hefx (moduli q < 2^30, residues held in uint32).
//
// The paper's reductions (Alg. 1 Montgomery on 16-bit primitives, Alg. 4 Barrett) were
// shaped for the TPU's 32-bit VPU.  On sm_103a the CUDA cores have a native 32x32->64-bit
// multiply (IMAD.WIDE / IMAD.HI), so the same reductions collapse to a few instructions:
//  - Shoup multiplication by a precomputed constant w (companion floor(w 2^32 / q)),
//    the form the twiddle products take (the "BUILD-option" Shoup reduction of Sec. V-G);
//  - Montgomery REDC (Alg. 1's postcondition: result = z 2^-32 mod q in [0, 2q)) for the
//    Hadamard product of two runtime residues;
//  - lazy ranges [0, 2q) / [0, 4q) along a chain with one final correction (App. C).
#pragma once
#include <cstdint>

namespace hefx {

// x * w mod q for constant w with Shoup companion wp; any x < 2^32; result in [0, 2q).
__device__ __forceinline__ uint32_t mul_shoup_lazy(uint32_t x, uint32_t w, uint32_t wp, uint32_t q) {
    uint32_t quot = __umulhi(x, wp);
    return x * w - quot * q;
}

// Montgomery REDC of x * y (x < 4q, y < q): returns x y 2^-32 mod q in [0, 2q).
__device__ __forceinline__ uint32_t mul_mont_lazy(uint32_t x, uint32_t y, uint32_t q, uint32_t qinv_neg) {
    uint64_t z = (uint64_t)x * y;
    uint32_t lo = (uint32_t)z, hi = (uint32_t)(z >> 32);
    uint32_t m = lo * qinv_neg;
    return hi + __umulhi(m, q) + (lo != 0u);
}

// x >= bound ? x - bound : x, as one unsigned min (x - bound wraps above x when x < bound).
__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t bound) { return umin(x, x - bound); }

// [0, 4q) -> [0, q)
__device__ __forceinline__ uint32_t reduce4(uint32_t x, uint32_t q) { return csub(csub(x, 2 * q), q); }

// Harvey's lazy Cooley-Tukey butterfly: x, y in [0, 4q) -> x + w y, x - w y in [0, 4q).
__device__ __forceinline__ void ct_bfly(uint32_t& x, uint32_t& y, uint32_t w, uint32_t wp, uint32_t q) {
    uint32_t two_q = 2 * q;
    uint32_t a = csub(x, two_q);
    uint32_t t = mul_shoup_lazy(y, w, wp, q);
    x = a + t;
    y = a - t + two_q;
}

// Lazy Gentleman-Sande butterfly: x, y in [0, 2q) -> x + y, (x - y) w in [0, 2q).
__device__ __forceinline__ void gs_bfly(uint32_t& x, uint32_t& y, uint32_t w, uint32_t wp, uint32_t q) {
    uint32_t two_q = 2 * q;
    uint32_t s = csub(x + y, two_q);
    uint32_t d = x - y + two_q;
    x = s;
    y = mul_shoup_lazy(d, w, wp, q);
}

}  // namespace hefx
