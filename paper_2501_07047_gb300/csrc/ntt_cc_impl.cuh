// CUDA-core negacyclic NTT / INTT (path a): radix-2 Cooley-Tukey forward and
// Gentleman-Sande inverse (App. A, "Radix-2 Cooley-Tukey NTT"; the garbled loop indices of
// the printed algorithm are replaced by the textbook ones), with lazy Shoup butterflies.
//
// GB300 mapping
//  - A row (one limb of one polynomial) is held in shared memory by one CTA (N <= 2^15) or
//    split over a cluster of P CTAs (P = 8 at N = 2^16: 32 KiB + padding and 128 threads
//    per CTA, registers sized for five CTAs of different rows per SM, so that their load,
//    compute and barrier phases overlap).  Each row is read from and written to HBM once
//    per transform (512 KiB per N = 2^16 limb-NTT).  A CTA with N < 2^13 holds 2^13 / N
//    rows.
//  - With P > 1 the log2(P) stages whose butterflies pair elements of different CTAs run
//    as one radix-P step through distributed shared memory: the forward transform computes
//    them while loading (each position j' of the first N/P is owned by one thread of the
//    cluster, which reads the P inputs j' + t N/P from global memory and stores output t
//    into CTA t's shared memory); the inverse computes them last, reading the P CTAs'
//    shared memory and writing global memory.
//  - The other stages run in register passes of up to 5 stages (radix-32 sub-transforms);
//    each pass reads and writes shared memory once, in a swizzled layout (swz) where both
//    strided and contiguous (uint4) sub-transform accesses are bank-conflict free.
//  - The forward output is in bit-reversed order with no shuffle (the twiddle table is
//    stored in bit-reversed order, as MAT folds permutations into constants, Sec. IV-B).
#pragma once
#include <cooperative_groups.h>

#include <algorithm>

#include "hefx_internal.h"
#include "modarith.cuh"
#include "tc_common.cuh"

namespace cg = cooperative_groups;

namespace hefx {
namespace cc {

// Shared-memory word of element j: the 16-byte chunk index within each 32-word row is XORed
// with the row's low three bits.  Consecutive elements (the strided passes' lanes) stay in
// one row, and 16-byte groups of the contiguous sub-transforms (read and written as uint4)
// of eight consecutive rows land on different banks: both patterns are conflict free.
__device__ __forceinline__ int swz(int j) { return j ^ (((j >> 5) & 7) << 2); }

// Word of element j0 + (k << logs) (k < 2^R) of a register pass's sub-transform in the
// swizzled buffer, j0 = row * m + jb the sub-transform's first element.  Equal to
// swz(j0 + (k << logs)) under each branch's condition, but written so that the per-element
// part is a compile-time offset (logs >= 8), one XOR with a constant (logs == 5: bits 5-7 of
// j0 are zero for one-row CTAs and R >= 3), or one XOR per 16-byte chunk (logs == 0: the
// sub-transform is 2^R-aligned inside one 32-word row).
template <int R, int logs, int ROWS>
__device__ __forceinline__ int swz_elem(int j0, int k) {
    if constexpr (logs >= 8) {
        return swz(j0) + (k << logs);
    } else if constexpr (logs == 5 && R >= 3 && ROWS == 1) {
        return (j0 ^ ((k & 7) << 2)) + (k << 5);
    } else if constexpr (logs == 0 && R >= 2 && R <= 5) {
        return (j0 & ~31) + (k ^ ((j0 & 31) ^ (((j0 >> 5) & 7) << 2)));
    } else {
        return swz(j0 + (k << logs));
    }
}

// Tuning knobs: log2 of the CTAs per row at N = 2^17 .. 2^14 (2^13 elements per CTA below
// N = 2^17), the threads of a CTA that holds less than 2^15 elements of a split row, and the
// CTAs per SM its register budget is sized for (N = 2^17: 2^14 elements and 64 KiB per CTA).
#ifndef HEFX_CC_LOGP17
#define HEFX_CC_LOGP17 3
#endif
#ifndef HEFX_CC_THREADS17
#define HEFX_CC_THREADS17 256
#endif
#ifndef HEFX_CC_MINB17
#define HEFX_CC_MINB17 2
#endif
#ifndef HEFX_CC_LOGP16
#define HEFX_CC_LOGP16 3
#endif
#ifndef HEFX_CC_LOGP15
#define HEFX_CC_LOGP15 2
#endif
#ifndef HEFX_CC_LOGP14
#define HEFX_CC_LOGP14 1
#endif
#ifndef HEFX_CC_SPLIT_THREADS
#define HEFX_CC_SPLIT_THREADS 128
#endif
#ifndef HEFX_CC_SPLIT_MINB
#define HEFX_CC_SPLIT_MINB 5
#endif
// log2 of the sub-transforms a thread of a one-row CTA runs together in a strided register
// pass (0: one at a time), for the split-row per-size kernels and for the fused batch kernel
// (one-CTA rows of 2^13 take pairs), and the kernel modes (bit 1 << MODE) that do so.
// Measured on config 2 (fwd + inv, us per step): 99.0 serialized / 74.0 pipelined with
// pairs, 96.1 / 72.3 with quads; one-CTA rows of 2^13 lost 3 % with quads; the fused product
// (NTT, Hadamard and INTT in one kernel, whose registers it crowds) is slower with either,
// and the batch kernel, which holds every ring degree's passes, keeps pairs.
#ifndef HEFX_CC_LOGPW
#define HEFX_CC_LOGPW 2
#endif
#ifndef HEFX_CC_LOGPW_BATCH
#define HEFX_CC_LOGPW_BATCH 1
#endif
#ifndef HEFX_CC_WIDE_MODES
#define HEFX_CC_WIDE_MODES 0x1b
#endif

// F & 16 selects the configuration of the fused batch kernel (every ring degree in CTAs of
// 128 threads and 2^13 elements, clusters of 8: one row of 2^16, two of 2^15, four of 2^14, or
// eight CTA-sized groups of smaller rows per cluster).
template <int LOGN, int F = 0>
struct Cfg {
    static constexpr int logP =
        LOGN >= 17   ? HEFX_CC_LOGP17
        : LOGN == 16 ? HEFX_CC_LOGP16
        : LOGN == 15 ? HEFX_CC_LOGP15
        : LOGN == 14 ? HEFX_CC_LOGP14
                     : 0;
    static constexpr int P = 1 << logP;  // CTAs (one cluster) per row
    static constexpr bool split = P > 1;
    static constexpr int logm = LOGN - logP;  // elements of one row segment
    static constexpr int m = 1 << logm;
    static constexpr int rows = (split || logm >= 13) ? 1 : (1 << (13 - logm));  // row segments per CTA
    static constexpr int elems = m * rows;
    static constexpr bool small_split = split && m < (1 << 15);
    static constexpr bool unified = (F & 16) != 0;
    static constexpr int threads = unified        ? 128
                                   : LOGN >= 17   ? HEFX_CC_THREADS17
                                   : small_split ? HEFX_CC_SPLIT_THREADS : (elems >= (1 << 14) ? 512 : 256);
    static constexpr int minb = unified ? 5 : LOGN >= 17 ? HEFX_CC_MINB17 : small_split ? HEFX_CC_SPLIT_MINB : 1;
    static constexpr int smem_bytes = elems * 4;
    static constexpr int S = logm;                  // stages run inside the CTA
    static constexpr int r_small = S < 5 ? S : 5;   // pass over the smallest strides
    static constexpr int rest = S - r_small;
    static constexpr int nrest = (rest + 4) / 5;
    __host__ __device__ static constexpr int big(int i) {
        return nrest == 0 ? 0 : rest / nrest + (i < rest % nrest ? 1 : 0);
    }
    static_assert(!split || (m / P) % threads == 0, "cross-CTA positions divide among the threads");
    static_assert(P <= 8, "portable cluster sizes only");
    static_assert(threads >= 128, "at least four warps per CTA");
};

struct KArgs {
    // the input viewed as [rows * N / 32][32] uint32, 128-byte swizzle, box 32 x 256: the
    // inverse transforms of the contiguous layout load their part of a row with it (TMA)
    alignas(64) CUtensorMap tmap_in;
    CUtensorMap tmap_out;  // the output, same view: forward transforms store their part with it
    uint32_t* err;      // bounded-wait error flag (a device word, 0 = no error)
    const uint32_t* in;
    const uint32_t* had;
    uint32_t* out;
    const uint2* tw_f;  // forward twiddles [L][N]
    const uint2* tw_i;  // inverse twiddles [L][N]
    const LimbConst* lc;
    const RowDesc* desc;  // per-row pointers and limb (batched jobs), or null: [rows][N] layout
    uint32_t rows;
    uint32_t L;
    uint32_t in_rows;  // MODE_RS_FWD: input rows per polynomial (the output has L = in_rows - 1)
};

// Row r's input / Hadamard operand / output and limb, from the descriptor list when there
// is one, else from the contiguous [batch][L][N] layout.
// F is a compile-time switch so that the contiguous-layout kernels carry no descriptor code.
template <int N, int F>
__device__ __forceinline__ const uint32_t* row_in(const KArgs& a, uint32_t r) {
    if constexpr ((F & 1) != 0) return a.desc[r].in;
    else return a.in + (size_t)r * N;
}
template <int N, int F>
__device__ __forceinline__ const uint32_t* row_had(const KArgs& a, uint32_t r) {
    if constexpr ((F & 1) != 0) return a.desc[r].had;
    else return a.had + (size_t)r * N;
}
template <int N, int F>
__device__ __forceinline__ uint32_t* row_out(const KArgs& a, uint32_t r) {
    if constexpr ((F & 1) != 0) return a.desc[r].out;
    else return a.out + (size_t)r * N;
}
template <int F>
__device__ __forceinline__ uint32_t row_limb(const KArgs& a, uint32_t r) {
    if constexpr ((F & 1) != 0) return a.desc[r].limb;
    else return r % a.L;
}
// Row r's limb constants and twiddle tables: from its descriptor (which carries its own
// parameter set's tables, so rows of different ring degrees can share a launch), else from the
// launch's parameter set.
template <int F>
__device__ __forceinline__ const LimbConst& row_lc(const KArgs& a, uint32_t r) {
    if constexpr ((F & 1) != 0) return *a.desc[r].lc;
    else return a.lc[r % a.L];
}
template <int N, int F>
__device__ __forceinline__ const uint2* row_twf(const KArgs& a, uint32_t r) {
    if constexpr ((F & 1) != 0) return a.desc[r].twf;
    else return a.tw_f + (size_t)(r % a.L) * N;
}
template <int N, int F>
__device__ __forceinline__ const uint2* row_twi(const KArgs& a, uint32_t r) {
    if constexpr ((F & 1) != 0) return a.desc[r].twi;
    else return a.tw_i + (size_t)(r % a.L) * N;
}
// A Hadamard operand load: the fused batch kernel (F & 16) reads operands written earlier in the
// same launch, so it takes the coherent path (L2) instead of the read-only one.
template <int F, typename T>
__device__ __forceinline__ T ld_had(const T* p) {
    if constexpr ((F & 16) != 0) return __ldcg(p);
    else return __ldg(p);
}

// Where a register pass takes its inputs and puts its outputs.
enum : int { SRC_SMEM = 0, SRC_GLOBAL = 1, SRC_GLOBAL_HAD = 3 };
enum : int { DST_SMEM = 0, DST_GLOBAL = 1, DST_GLOBAL_REDUCE = 2, DST_SMEM_REDUCE = 3 };

// The CTA's share of the batch: rows [row0, row0 + nrows), or segment `part` (elements
// [gbase, gbase + m)) of row row0 when the row is split.
struct Seg {
    uint32_t row0, gbase, part;
    int nrows;
    uint32_t rbase;  // cluster rank of the row's first CTA (the fused batch kernel runs several rows per cluster)
};

// Canonical value of a forward output: from [0, 4q) (Harvey ranges) or [0, 16q) (lazy
// ranges, reduced to [0, 2q) by a Shoup product with 1 first).
template <int F>
__device__ __forceinline__ uint32_t reduce_out(uint32_t x, const LimbConst& lc) {
    if constexpr ((F & 2) != 0) return csub(mul_shoup_lazy(x, 1u, lc.one_sh, lc.q), lc.q);
    return csub(csub(x, 2 * lc.q), lc.q);
}

// Loads the 2^R elements jb + k * 2^logs (k < 2^R) of local row `row` into x.
template <int R, int LOGN, int logs, int SRC, int F>
__device__ __forceinline__ void load_elems(uint32_t (&x)[1 << R], const uint32_t* sm, const KArgs& a, const Seg& sg,
                                           int row, int jb, const LimbConst& lc) {
    using C = Cfg<LOGN, F>;
    constexpr int N = 1 << LOGN;
    if constexpr (SRC == SRC_SMEM) {
        const int j0 = row * C::m + jb;
        if constexpr (logs == 0 && R >= 2) {
#pragma unroll
            for (int k = 0; k < (1 << R); k += 4) {
                const uint4 v = *reinterpret_cast<const uint4*>(&sm[swz_elem<R, logs, C::rows>(j0, k)]);
                x[k] = v.x;
                x[k + 1] = v.y;
                x[k + 2] = v.z;
                x[k + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < (1 << R); ++k) x[k] = sm[swz_elem<R, logs, C::rows>(j0, k)];
        }
    } else {
        const bool valid = row < sg.nrows;
        const uint32_t grow_r = valid ? sg.row0 + row : sg.row0;
        const uint32_t* rin = row_in<N, F>(a, grow_r);
        const uint32_t* rhad = SRC == SRC_GLOBAL_HAD ? row_had<N, F>(a, grow_r) : nullptr;
        if constexpr (logs == 0 && R >= 2) {
            const uint4* src = reinterpret_cast<const uint4*>(rin + sg.gbase + jb);
            const uint4* hs = reinterpret_cast<const uint4*>(rhad + sg.gbase + jb);
#pragma unroll
            for (int k = 0; k < (1 << R); k += 4) {
                uint4 v = valid ? ld_had<F>(src + k / 4) : make_uint4(0, 0, 0, 0);
                if constexpr (SRC == SRC_GLOBAL_HAD) {
                    const uint4 h = valid ? ld_had<F>(hs + k / 4) : make_uint4(0, 0, 0, 0);
                    v.x = mul_mont_lazy(v.x, h.x, lc.q, lc.qinv_neg);
                    v.y = mul_mont_lazy(v.y, h.y, lc.q, lc.qinv_neg);
                    v.z = mul_mont_lazy(v.z, h.z, lc.q, lc.qinv_neg);
                    v.w = mul_mont_lazy(v.w, h.w, lc.q, lc.qinv_neg);
                }
                x[k] = v.x;
                x[k + 1] = v.y;
                x[k + 2] = v.z;
                x[k + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < (1 << R); ++k) {
                const size_t g = sg.gbase + jb + (k << logs);
                uint32_t v = valid ? ld_had<F>(rin + g) : 0u;
                if constexpr (SRC == SRC_GLOBAL_HAD) v = mul_mont_lazy(v, valid ? ld_had<F>(rhad + g) : 0u, lc.q, lc.qinv_neg);
                x[k] = v;
            }
        }
    }
}

template <int R, int LOGN, int logs, int DST, int F>
__device__ __forceinline__ void store_elems(const uint32_t (&x)[1 << R], uint32_t* sm, const KArgs& a, const Seg& sg,
                                            int row, int jb, const LimbConst& lc) {
    using C = Cfg<LOGN, F>;
    constexpr int N = 1 << LOGN;
    if constexpr (DST == DST_SMEM_REDUCE) {  // canonical values into the swizzled buffer (TMA store)
        static_assert(logs == 0 && R >= 2, "the smallest-stride pass");
        const int j0 = row * C::m + jb;
#pragma unroll
        for (int k = 0; k < (1 << R); k += 4)
            *reinterpret_cast<uint4*>(&sm[swz_elem<R, logs, C::rows>(j0, k)]) =
                make_uint4(reduce_out<F>(x[k], lc), reduce_out<F>(x[k + 1], lc), reduce_out<F>(x[k + 2], lc),
                           reduce_out<F>(x[k + 3], lc));
    } else if constexpr (DST == DST_SMEM) {
        const int j0 = row * C::m + jb;
        if constexpr (logs == 0 && R >= 2) {
#pragma unroll
            for (int k = 0; k < (1 << R); k += 4)
                *reinterpret_cast<uint4*>(&sm[swz_elem<R, logs, C::rows>(j0, k)]) =
                    make_uint4(x[k], x[k + 1], x[k + 2], x[k + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < (1 << R); ++k) sm[swz_elem<R, logs, C::rows>(j0, k)] = x[k];
        }
    } else {
        if (row >= sg.nrows) return;
        uint32_t* dst = row_out<N, F>(a, sg.row0 + row) + sg.gbase + jb;
        if constexpr (logs == 0 && R >= 2) {
#pragma unroll
            for (int k = 0; k < (1 << R); k += 4) {
                uint4 v = make_uint4(x[k], x[k + 1], x[k + 2], x[k + 3]);
                if constexpr (DST == DST_GLOBAL_REDUCE) {
                    v.x = reduce_out<F>(v.x, lc);
                    v.y = reduce_out<F>(v.y, lc);
                    v.z = reduce_out<F>(v.z, lc);
                    v.w = reduce_out<F>(v.w, lc);
                }
                reinterpret_cast<uint4*>(dst)[k / 4] = v;
            }
        } else {
#pragma unroll
            for (int k = 0; k < (1 << R); ++k) dst[k << logs] = DST == DST_GLOBAL_REDUCE ? reduce_out<F>(x[k], lc) : x[k];
        }
    }
}

// Lazy-range schedules for moduli below 2^28 (flag F & 2), where values may grow to
// 16q < 2^32.  A Shoup product with 1 (x - floor(x floor(2^32/q) / 2^32) q, two IMADs)
// brings any 32-bit value into [0, 2q); it replaces the conditional subtractions of
// Harvey's butterflies at the few stages where a bound (in units of q) would pass 16.
//  - forward (Cooley-Tukey): the first input enters stage s below fwd_bound_in(s) q; it is
//    reduced where fwd_bound_in(s) + 2 > 16, and the outputs are below (its bound + 2) q.
//  - inverse (Gentleman-Sande): both inputs of stage e are below inv_bound_in(e) q (2 for a
//    canonical or Montgomery-product input); the sum doubles the bound and is reduced where
//    it would pass 8 (so the next stage's sum and difference stay below 16q).
__host__ __device__ constexpr int fwd_bound_in(int s) {
    int b = 1;
    for (int t = 0; t < s; ++t) b = (b + 2 > 16 ? 2 : b) + 2;
    return b;
}
__host__ __device__ constexpr int inv_bound_in(int e) {
    int b = 2;
    for (int t = 0; t < e; ++t) b = 2 * b > 8 ? 2 : 2 * b;
    return b;
}

// Twiddle product x w mod q in [0, 2q) for any x < 2^32, by the reduction F selects (bits 2-3):
// 0 Shoup (w.y = floor(w 2^32 / q)), 1 Montgomery (w.x holds w 2^32 mod q; one REDC), 2 Barrett
// (64-bit product, quotient from floor(2^64 / q)).  The three are the variants of the paper's
// modular-reduction ablation (Sec. V-F); Shoup is the default.
template <int F>
__device__ __forceinline__ uint32_t twmul(uint32_t x, uint2 w, const LimbConst& lc) {
    constexpr int RED = (F >> 2) & 3;
    if constexpr (RED == 1) {
        return mul_mont_lazy(x, w.x, lc.q, lc.qinv_neg);
    } else if constexpr (RED == 2) {
        const uint64_t z = (uint64_t)x * w.x;
        const uint64_t mu = ((uint64_t)lc.bar_hi << 32) | lc.bar_lo;
        return (uint32_t)(z - __umul64hi(z, mu) * lc.q);
    } else {
        return mul_shoup_lazy(x, w.x, w.y, lc.q);
    }
}

// c q for the lazy inverse offsets (c = 2, 4 or 8), from the limb's constants.
__device__ __forceinline__ uint32_t q_multiple(const LimbConst& lc, int c) {
    return c == 2 ? lc.q2 : c == 4 ? lc.q4 : c == 8 ? lc.q8 : (uint32_t)c * lc.q;
}

// R forward (Cooley-Tukey) stages s0 .. s0+R-1 on registers; stage s pairs j, j + N/2^(s+1)
// and uses twiddle psi^brv(2^s + G) for group G (one load per group, reused by its
// butterflies).  Without F & 2 every butterfly keeps Harvey's [0, 4q) range (q < 2^30).
template <int R, int LOGN, int s0, int F>
__device__ __forceinline__ void fwd_stages(uint32_t (&x)[1 << R], uint32_t g0, const uint2* tw, const LimbConst& lc) {
    // the smallest-stride pass reads the group-major part of the table
    constexpr bool PERM = (s0 + R == LOGN);
    constexpr bool LAZY = (F & 2) != 0;
    const uint32_t q = lc.q, two_q = lc.q2;
#pragma unroll
    for (int v = 0; v < R; ++v) {
        const int half = 1 << (R - 1 - v);
        const bool corr = !LAZY || fwd_bound_in(s0 + v) + 2 > 16;
        uint2 w = make_uint2(0, 0);
        // one base pointer per stage: the loads below have compile-time offsets
        const uint2* base = PERM ? tw + g0 + (1u << (s0 + v)) : tw + (1u << (s0 + v)) + ((size_t)g0 << v);
#pragma unroll
        for (int b = 0; b < (1 << (R - 1)); ++b) {
            const int g = b >> (R - 1 - v);
            const int k = (g << (R - v)) + (b & (half - 1));
            if ((b & (half - 1)) == 0) w = __ldg(base + (PERM ? (g << s0) : g));
            const uint32_t xa = !corr ? x[k] : (LAZY ? mul_shoup_lazy(x[k], 1u, lc.one_sh, q) : csub(x[k], two_q));
            const uint32_t t = twmul<F>(x[k + half], w, lc);
            x[k] = xa + t;
            x[k + half] = xa - t + two_q;
        }
    }
}

// R inverse (Gentleman-Sande) stages e0 .. e0+R-1 on registers; stage e pairs j, j + 2^e with
// twiddle psi^-brv(N/2^(e+1) + G).  SCALE folds N^-1 (1) or N^-1 2^32 (2) into stage LOGN-1.
// Inputs are below 2q (canonical, or a Montgomery Hadamard product); outputs of the scaled
// stage are canonical.  Without F & 2 every butterfly keeps Harvey's [0, 2q) range.
template <int R, int LOGN, int SCALE, int e0, int F>
__device__ __forceinline__ void inv_stages(uint32_t (&x)[1 << R], uint32_t gbase, int j_hi, const uint2* tw,
                                           const LimbConst& lc) {
    constexpr int N = 1 << LOGN;
    constexpr bool PERM = (e0 == 0);  // the smallest-stride pass reads the group-major table part
    constexpr bool LAZY = (F & 2) != 0;
    const uint32_t q = lc.q, two_q = lc.q2;
    const uint32_t J = (gbase >> R) + (uint32_t)j_hi;  // global index of the sub-transform (e0 == 0)
#pragma unroll
    for (int v = 0; v < R; ++v) {
        const int e = e0 + v;
        const int h = 1 << v;
        // X - Y + c q >= 0 for Y below c q; the sum is reduced where its bound passes 8q
        const uint32_t cq = LAZY ? q_multiple(lc, inv_bound_in(e)) : two_q;
        const bool red = !LAZY || 2 * inv_bound_in(e) > 8;
        if (SCALE && e == LOGN - 1) {
            const uint32_t s = SCALE == 1 ? lc.ninv : lc.ninvR, ssh = SCALE == 1 ? lc.ninv_sh : lc.ninvR_sh;
            const uint32_t w = SCALE == 1 ? lc.ninvw : lc.ninvRw, wsh = SCALE == 1 ? lc.ninvw_sh : lc.ninvRw_sh;
#pragma unroll
            for (int kk = 0; kk < (1 << (R - 1)); ++kk) {
                const uint32_t X = x[kk], Y = x[kk + h];
                const uint32_t s0v = mul_shoup_lazy(X + Y, s, ssh, q), s1v = mul_shoup_lazy(X - Y + cq, w, wsh, q);
                x[kk] = csub(s0v, q);
                x[kk + h] = csub(s1v, q);
            }
            continue;
        }
        const uint2* base = PERM ? tw + (uint32_t)(N >> (e + 1)) + J
                                 : tw + (uint32_t)(N >> (e + 1)) + (gbase >> (e + 1)) + ((uint32_t)j_hi << (R - v - 1));
        uint2 w = make_uint2(0, 0);
#pragma unroll
        for (int b = 0; b < (1 << (R - 1)); ++b) {
            const int g = b >> v;
            const int k = (g << (v + 1)) + (b & (h - 1));
            if ((b & (h - 1)) == 0) w = __ldg(base + (PERM ? (g << (LOGN - R)) : g));
            const uint32_t X = x[k], Y = x[k + h];
            const uint32_t sum = X + Y;
            x[k] = !red ? sum : (LAZY ? mul_shoup_lazy(sum, 1u, lc.one_sh, q) : csub(sum, two_q));
            x[k + h] = twmul<F>(X - Y + cq, w, lc);
        }
    }
}

// Twiddles of R forward stages s0 .. s0+R-1 for one sub-transform, loaded up front:
// w[2^v - 1 + g] is stage s0+v's twiddle for group g (the ones fwd_stages loads one by one).
// The table is read through one base pointer per stage so that every load of a stage has a
// compile-time offset.
template <int R, int LOGN, int s0>
__device__ __forceinline__ void load_tw_fwd(uint2 (&w)[(1 << R) - 1], uint32_t g0, const uint2* tw) {
    constexpr bool PERM = (s0 + R == LOGN);
#pragma unroll
    for (int v = 0; v < R; ++v) {
        const uint2* base = PERM ? tw + g0 + (1u << (s0 + v)) : tw + (1u << (s0 + v)) + ((size_t)g0 << v);
#pragma unroll
        for (int g = 0; g < (1 << v); ++g) w[(1 << v) - 1 + g] = __ldg(base + (PERM ? (g << s0) : g));
    }
}

// fwd_stages on preloaded twiddles.
template <int R, int LOGN, int s0, int F>
__device__ __forceinline__ void fwd_stages_w(uint32_t (&x)[1 << R], const uint2 (&w)[(1 << R) - 1],
                                             const LimbConst& lc) {
    constexpr bool LAZY = (F & 2) != 0;
    const uint32_t q = lc.q, two_q = lc.q2;
#pragma unroll
    for (int v = 0; v < R; ++v) {
        const int half = 1 << (R - 1 - v);
        const bool corr = !LAZY || fwd_bound_in(s0 + v) + 2 > 16;
#pragma unroll
        for (int b = 0; b < (1 << (R - 1)); ++b) {
            const int g = b >> (R - 1 - v);
            const int k = (g << (R - v)) + (b & (half - 1));
            const uint32_t xa = !corr ? x[k] : (LAZY ? mul_shoup_lazy(x[k], 1u, lc.one_sh, q) : csub(x[k], two_q));
            const uint32_t t = twmul<F>(x[k + half], w[(1 << v) - 1 + g], lc);
            x[k] = xa + t;
            x[k + half] = xa - t + two_q;
        }
    }
}

// Offset of inverse stage v's twiddles in the preloaded array (stage v has 2^(R-1-v) groups).
__host__ __device__ constexpr int inv_tw_off(int R, int v) { return (1 << R) - (1 << (R - v)); }

// Twiddles of R inverse stages e0 .. e0+R-1 for one sub-transform (those inv_stages loads one
// by one; the scaled last stage takes its constants from LimbConst and has no entry).
template <int R, int LOGN, int SCALE, int e0>
__device__ __forceinline__ void load_tw_inv(uint2 (&w)[(1 << R) - 1], uint32_t gbase, int j_hi, const uint2* tw) {
    constexpr int N = 1 << LOGN;
    constexpr bool PERM = (e0 == 0);
    const uint32_t J = (gbase >> R) + (uint32_t)j_hi;
#pragma unroll
    for (int v = 0; v < R; ++v) {
        const int e = e0 + v;
        if (SCALE && e == LOGN - 1) continue;
        const uint2* base = PERM ? tw + (uint32_t)(N >> (e + 1)) + J
                                 : tw + (uint32_t)(N >> (e + 1)) + (gbase >> (e + 1)) + ((uint32_t)j_hi << (R - v - 1));
#pragma unroll
        for (int g = 0; g < (1 << (R - 1 - v)); ++g)
            w[inv_tw_off(R, v) + g] = __ldg(base + (PERM ? (g << (LOGN - R)) : g));
    }
}

// inv_stages on preloaded twiddles.
template <int R, int LOGN, int SCALE, int e0, int F>
__device__ __forceinline__ void inv_stages_w(uint32_t (&x)[1 << R], const uint2 (&w)[(1 << R) - 1],
                                             const LimbConst& lc) {
    constexpr bool LAZY = (F & 2) != 0;
    const uint32_t q = lc.q, two_q = lc.q2;
#pragma unroll
    for (int v = 0; v < R; ++v) {
        const int e = e0 + v;
        const int h = 1 << v;
        const uint32_t cq = LAZY ? q_multiple(lc, inv_bound_in(e)) : two_q;
        const bool red = !LAZY || 2 * inv_bound_in(e) > 8;
        if (SCALE && e == LOGN - 1) {
            const uint32_t s = SCALE == 1 ? lc.ninv : lc.ninvR, ssh = SCALE == 1 ? lc.ninv_sh : lc.ninvR_sh;
            const uint32_t wv = SCALE == 1 ? lc.ninvw : lc.ninvRw, wsh = SCALE == 1 ? lc.ninvw_sh : lc.ninvRw_sh;
#pragma unroll
            for (int kk = 0; kk < (1 << (R - 1)); ++kk) {
                const uint32_t X = x[kk], Y = x[kk + h];
                const uint32_t s0v = mul_shoup_lazy(X + Y, s, ssh, q), s1v = mul_shoup_lazy(X - Y + cq, wv, wsh, q);
                x[kk] = csub(s0v, q);
                x[kk + h] = csub(s1v, q);
            }
            continue;
        }
#pragma unroll
        for (int b = 0; b < (1 << (R - 1)); ++b) {
            const int g = b >> v;
            const int k = (g << (v + 1)) + (b & (h - 1));
            const uint32_t X = x[k], Y = x[k + h];
            const uint32_t sum = X + Y;
            x[k] = !red ? sum : (LAZY ? mul_shoup_lazy(sum, 1u, lc.one_sh, q) : csub(sum, two_q));
            x[k + h] = twmul<F>(X - Y + cq, w[inv_tw_off(R, v) + g], lc);
        }
    }
}

// Flag bit of F, set by run_task for the passes of the modes in HEFX_CC_WIDE_MODES: the
// strided passes run 2^HEFX_CC_LOGPW (batch kernel: 2^HEFX_CC_LOGPW_BATCH; one-CTA rows: 2)
// sub-transforms per thread together.
constexpr int kWide = 32;

// The 2^LW adjacent sub-transforms j0, j0 + 1, ... (j0 a multiple of 2^LW, smallest stride
// 2^logs >= 2^LW) of a strided pass, element k of all of them as one 8- or 16-byte access: the
// swizzle permutes 16-byte chunks only, so the 2^LW words stay adjacent and aligned.
template <int R, int LW, int logs, int ROWS>
__device__ __forceinline__ void load_wide(uint32_t (&x)[1 << LW][1 << R], const uint32_t* sm, int j0) {
    static_assert(LW == 1 || LW == 2, "pairs or quads");
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        const uint32_t* p = &sm[swz_elem<R, logs, ROWS>(j0, k)];
        if constexpr (LW == 1) {
            const uint2 v = *reinterpret_cast<const uint2*>(p);
            x[0][k] = v.x;
            x[1][k] = v.y;
        } else {
            const uint4 v = *reinterpret_cast<const uint4*>(p);
            x[0][k] = v.x;
            x[1][k] = v.y;
            x[2][k] = v.z;
            x[3][k] = v.w;
        }
    }
}
template <int R, int LW, int logs, int ROWS>
__device__ __forceinline__ void store_wide(const uint32_t (&x)[1 << LW][1 << R], uint32_t* sm, int j0) {
#pragma unroll
    for (int k = 0; k < (1 << R); ++k) {
        uint32_t* p = &sm[swz_elem<R, logs, ROWS>(j0, k)];
        if constexpr (LW == 1) *reinterpret_cast<uint2*>(p) = make_uint2(x[0][k], x[1][k]);
        else *reinterpret_cast<uint4*>(p) = make_uint4(x[0][k], x[1][k], x[2][k], x[3][k]);
    }
}

// Forward register pass over stages s0 .. s0+R-1 of every sub-transform of the CTA.
template <int R, int LOGN, int s0, int SRC, int DST, int F>
__device__ __forceinline__ void fwd_pass(uint32_t* sm, const Seg& sg, const KArgs& a) {
    using C = Cfg<LOGN, F>;
    constexpr int N = 1 << LOGN;
    constexpr int logtl = LOGN - s0 - R;  // log2 of the smallest stride of the pass
    constexpr int lognsub = C::logm - R;
    constexpr int nsub = 1 << lognsub;
    constexpr int LW = (F & kWide) ? (C::unified ? HEFX_CC_LOGPW_BATCH : C::split ? HEFX_CC_LOGPW : 1) : 0;
    if constexpr (R <= 4 && C::rows == 1 && LW > 0 && logtl >= LW && SRC == SRC_SMEM && DST == DST_SMEM) {
        // one row, shared memory in and out: a thread runs the 2^LW sub-transforms j_lo ..
        // j_lo + 2^LW - 1 together (same group, so the same twiddles, loaded once)
        const LimbConst& lc = row_lc<F>(a, sg.row0);
        const uint2* tw = row_twf<N, F>(a, sg.row0);
        constexpr bool ONE = logtl >= lognsub;  // every sub-transform of the CTA in one group
        uint2 w[(1 << R) - 1];
        if constexpr (ONE) load_tw_fwd<R, LOGN, s0>(w, sg.gbase >> (logtl + R), tw);
#pragma unroll 1
        for (int u = threadIdx.x; u < (nsub >> LW); u += C::threads) {
            const int j_lo = (u & ((1 << (logtl - LW)) - 1)) << LW;
            const int j_hi = u >> (logtl - LW);
            if constexpr (!ONE) load_tw_fwd<R, LOGN, s0>(w, (sg.gbase >> (logtl + R)) + (uint32_t)j_hi, tw);
            const int jb = (j_hi << (logtl + R)) + j_lo;
            uint32_t x[1 << LW][1 << R];
            load_wide<R, LW, logtl, C::rows>(x, sm, jb);
#pragma unroll
            for (int c = 0; c < (1 << LW); ++c) fwd_stages_w<R, LOGN, s0, F>(x[c], w, lc);
            store_wide<R, LW, logtl, C::rows>(x, sm, jb);
        }
    } else if constexpr (R <= 4 && C::rows == 1) {
        // one row: every sub-transform shares the limb; each sub-transform's twiddles are all
        // requested before its data is read, so their latency is paid once per sub-transform
        // rather than once per stage
        const LimbConst& lc = row_lc<F>(a, sg.row0);
        const uint2* tw = row_twf<N, F>(a, sg.row0);
#pragma unroll 1
        for (int u = threadIdx.x; u < nsub; u += C::threads) {
            uint2 w[(1 << R) - 1];
            load_tw_fwd<R, LOGN, s0>(w, (sg.gbase >> (logtl + R)) + (uint32_t)(u >> logtl), tw);
            const int j_lo = u & ((1 << logtl) - 1);
            const int j_hi = u >> logtl;
            const int jb = (j_hi << (logtl + R)) + j_lo;
            uint32_t x[1 << R];
            load_elems<R, LOGN, logtl, SRC, F>(x, sm, a, sg, 0, jb, lc);
            fwd_stages_w<R, LOGN, s0, F>(x, w, lc);
            store_elems<R, LOGN, logtl, DST, F>(x, sm, a, sg, 0, jb, lc);
        }
    } else {
        for (int u = threadIdx.x; u < C::rows * nsub; u += C::threads) {
            const int row = C::rows == 1 ? 0 : u >> lognsub;
            const int uu = u & (nsub - 1);
            const int j_lo = uu & ((1 << logtl) - 1);
            const int j_hi = uu >> logtl;
            const int jb = (j_hi << (logtl + R)) + j_lo;
            const uint32_t g0 = (sg.gbase >> (logtl + R)) + (uint32_t)j_hi;
            const uint32_t rr = row < sg.nrows ? sg.row0 + row : sg.row0;
            const LimbConst& lc = row_lc<F>(a, rr);
            const uint2* tw = row_twf<N, F>(a, rr);
            uint32_t x[1 << R];
            load_elems<R, LOGN, logtl, SRC, F>(x, sm, a, sg, row, jb, lc);
            fwd_stages<R, LOGN, s0, F>(x, g0, tw, lc);
            store_elems<R, LOGN, logtl, DST, F>(x, sm, a, sg, row, jb, lc);
        }
    }
}

// Inverse register pass over stages e0 .. e0+R-1.
template <int R, int LOGN, int SCALE, int e0, int SRC, int DST, int F>
__device__ __forceinline__ void inv_pass(uint32_t* sm, const Seg& sg, const KArgs& a) {
    using C = Cfg<LOGN, F>;
    constexpr int N = 1 << LOGN;
    constexpr int lognsub = C::logm - R;
    constexpr int nsub = 1 << lognsub;
    constexpr int LW = (F & kWide) ? (C::unified ? HEFX_CC_LOGPW_BATCH : C::split ? HEFX_CC_LOGPW : 1) : 0;
    if constexpr (R <= 4 && C::rows == 1 && LW > 0 && e0 >= LW && SRC == SRC_SMEM && DST == DST_SMEM) {
        // as fwd_pass: 2^LW adjacent sub-transforms per thread, one twiddle set
        const LimbConst& lc = row_lc<F>(a, sg.row0);
        const uint2* tw = row_twi<N, F>(a, sg.row0);
        constexpr bool ONE = e0 >= lognsub;  // every sub-transform of the CTA in one group
        uint2 w[(1 << R) - 1];
        if constexpr (ONE) load_tw_inv<R, LOGN, SCALE, e0>(w, sg.gbase, 0, tw);
#pragma unroll 1
        for (int u = threadIdx.x; u < (nsub >> LW); u += C::threads) {
            const int j_lo = (u & ((1 << (e0 - LW)) - 1)) << LW;
            const int j_hi = u >> (e0 - LW);
            if constexpr (!ONE) load_tw_inv<R, LOGN, SCALE, e0>(w, sg.gbase, j_hi, tw);
            const int jb = (j_hi << (e0 + R)) + j_lo;
            uint32_t x[1 << LW][1 << R];
            load_wide<R, LW, e0, C::rows>(x, sm, jb);
#pragma unroll
            for (int c = 0; c < (1 << LW); ++c) inv_stages_w<R, LOGN, SCALE, e0, F>(x[c], w, lc);
            store_wide<R, LW, e0, C::rows>(x, sm, jb);
        }
    } else if constexpr (R <= 4 && C::rows == 1) {
        // as fwd_pass: a sub-transform's twiddles are all requested before its data is read
        const LimbConst& lc = row_lc<F>(a, sg.row0);
        const uint2* tw = row_twi<N, F>(a, sg.row0);
#pragma unroll 1
        for (int u = threadIdx.x; u < nsub; u += C::threads) {
            uint2 w[(1 << R) - 1];
            load_tw_inv<R, LOGN, SCALE, e0>(w, sg.gbase, u >> e0, tw);
            const int j_lo = u & ((1 << e0) - 1);
            const int j_hi = u >> e0;
            const int jb = (j_hi << (e0 + R)) + j_lo;
            uint32_t x[1 << R];
            load_elems<R, LOGN, e0, SRC, F>(x, sm, a, sg, 0, jb, lc);
            inv_stages_w<R, LOGN, SCALE, e0, F>(x, w, lc);
            store_elems<R, LOGN, e0, DST, F>(x, sm, a, sg, 0, jb, lc);
        }
    } else {
        for (int u = threadIdx.x; u < C::rows * nsub; u += C::threads) {
            const int row = C::rows == 1 ? 0 : u >> lognsub;
            const int uu = u & (nsub - 1);
            const int j_lo = uu & ((1 << e0) - 1);
            const int j_hi = uu >> e0;
            const int jb = (j_hi << (e0 + R)) + j_lo;
            const uint32_t rr = row < sg.nrows ? sg.row0 + row : sg.row0;
            const LimbConst& lc = row_lc<F>(a, rr);
            const uint2* tw = row_twi<N, F>(a, rr);
            uint32_t x[1 << R];
            load_elems<R, LOGN, e0, SRC, F>(x, sm, a, sg, row, jb, lc);
            inv_stages<R, LOGN, SCALE, e0, F>(x, sg.gbase, j_hi, tw, lc);
            store_elems<R, LOGN, e0, DST, F>(x, sm, a, sg, row, jb, lc);
        }
    }
}

// The polynomial product's middle: the forward pass over the smallest strides, the Hadamard
// product with `had` (Montgomery, 2^-32 folded into the final scale) and the inverse pass
// over the same strides, on the same registers.
template <int R, int LOGN, int s0, int SRC, int DST, int F>
__device__ __forceinline__ void fwd_had_inv_pass(uint32_t* sm, const Seg& sg, const KArgs& a) {
    using C = Cfg<LOGN, F>;
    constexpr int N = 1 << LOGN;
    constexpr int lognsub = C::logm - R;
    constexpr int nsub = 1 << lognsub;
    static_assert(LOGN - s0 - R == 0, "the fused pass covers the smallest strides");
    for (int u = threadIdx.x; u < C::rows * nsub; u += C::threads) {
        const int row = C::rows == 1 ? 0 : u >> lognsub;
        const int j_hi = u & (nsub - 1);
        const int jb = j_hi << R;
        const uint32_t g0 = (sg.gbase >> R) + (uint32_t)j_hi;
        const uint32_t rr = row < sg.nrows ? sg.row0 + row : sg.row0;
        const LimbConst& lc = row_lc<F>(a, rr);
        uint32_t x[1 << R];
        load_elems<R, LOGN, 0, SRC, F>(x, sm, a, sg, row, jb, lc);
        fwd_stages<R, LOGN, s0, F>(x, g0, row_twf<N, F>(a, rr), lc);
        const bool valid = row < sg.nrows;
        const uint4* hs = reinterpret_cast<const uint4*>(row_had<N, F>(a, valid ? sg.row0 + row : sg.row0) + sg.gbase + jb);
#pragma unroll
        for (int k = 0; k < (1 << R); k += 4) {
            const uint4 h = valid ? ld_had<F>(hs + k / 4) : make_uint4(0, 0, 0, 0);
            x[k] = mul_mont_lazy(x[k], h.x, lc.q, lc.qinv_neg);
            x[k + 1] = mul_mont_lazy(x[k + 1], h.y, lc.q, lc.qinv_neg);
            x[k + 2] = mul_mont_lazy(x[k + 2], h.z, lc.q, lc.qinv_neg);
            x[k + 3] = mul_mont_lazy(x[k + 3], h.w, lc.q, lc.qinv_neg);
        }
        inv_stages<R, LOGN, 2, 0, F>(x, sg.gbase, j_hi, row_twi<N, F>(a, rr), lc);
        store_elems<R, LOGN, 0, DST, F>(x, sm, a, sg, row, jb, lc);
    }
}

// 32-bit address of this CTA's shared-memory word `sm` in cluster rank t's shared memory
// (shared::cluster window), and loads / stores through such addresses.
__device__ __forceinline__ uint32_t cluster_addr(const uint32_t* sm, uint32_t t) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(sm)), "r"(t));
    return r;
}
__device__ __forceinline__ void st_cluster4(uint32_t addr, uint4 v) {
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ uint4 ld_cluster4(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

template <bool SPLIT>
__device__ __forceinline__ void sync_all() {
    if constexpr (SPLIT) cg::this_cluster().sync();
    else __syncthreads();
}

// Forward passes I .. nrest-1 (big strides), SMEM -> SMEM; the first reads global memory
// unless the cross-CTA stages already filled shared memory.
template <int LOGN, int I, int s, int F>
__device__ __forceinline__ void fwd_big(uint32_t* sm, const Seg& sg, const KArgs& a) {
    using C = Cfg<LOGN, F>;
    if constexpr (I < C::nrest) {
        constexpr int r = C::big(I);
        constexpr int SRC = (I == 0 && !C::split) ? SRC_GLOBAL : SRC_SMEM;
        fwd_pass<r, LOGN, s, SRC, DST_SMEM, F>(sm, sg, a);
        __syncthreads();
        fwd_big<LOGN, I + 1, s + r, F>(sm, sg, a);
    }
}

// Inverse passes over big strides, from I down to 0; the last one writes global memory
// unless the row is split (then the cross-CTA stages follow).
template <int LOGN, int SCALE, int I, int e, int F>
__device__ __forceinline__ void inv_big(uint32_t* sm, const Seg& sg, const KArgs& a) {
    using C = Cfg<LOGN, F>;
    if constexpr (I >= 0) {
        constexpr int r = C::big(I);
        if constexpr (I == 0 && !C::split) {
            inv_pass<r, LOGN, SCALE, e, SRC_SMEM, DST_GLOBAL, F>(sm, sg, a);
        } else {
            inv_pass<r, LOGN, C::split ? 0 : SCALE, e, SRC_SMEM, DST_SMEM, F>(sm, sg, a);
            __syncthreads();
            inv_big<LOGN, SCALE, I - 1, e + r, F>(sm, sg, a);
        }
    }
}

// x_i -> (x_i - [x_{L-1}]_{q_i}) q_{L-1}^-1 mod q_i (Rescale by the set's last prime; canonical).
__device__ __forceinline__ uint32_t rescale_one(uint32_t x, uint32_t last_raw, const LimbConst& c) {
    const uint32_t last = csub(mul_shoup_lazy(last_raw, 1u, c.one_sh, c.q), c.q);
    return csub(mul_shoup_lazy(x + c.q - last, c.rs_inv, c.rs_inv_sh, c.q), c.q);
}

// Forward stages 0 .. logP-1 of a split row, whose butterflies pair elements of different
// CTAs: position j' < N/P is owned by one thread of the cluster (four consecutive positions
// per thread, moved as uint4), which reads the P inputs j' + t N/P from global memory, runs
// the radix-P step and stores output t into CTA t's shared memory.  Ends with a cluster
// barrier (outputs visible; every global read of the row done before any CTA writes it,
// so in-place transforms are safe).

template <int LOGN, int F, bool RS = false>
__device__ __forceinline__ void fwd_cross_pass(uint32_t* sm, const Seg& sg, const KArgs& a) {
    using C = Cfg<LOGN, F>;
    constexpr int N = 1 << LOGN, P = C::P, share = C::m / P, ITERS = share / (4 * C::threads);
    static_assert(share % (4 * C::threads) == 0, "whole uint4 groups per thread");
    uint32_t dst[P];
#pragma unroll
    for (int t = 0; t < P; ++t) dst[t] = cluster_addr(sm, sg.rbase + t);
    const uint32_t limb = row_limb<F>(a, sg.row0);
    const LimbConst& lc = row_lc<F>(a, sg.row0);
    const uint2* tw = row_twf<N, F>(a, sg.row0);
    const uint32_t* rin = row_in<N, F>(a, sg.row0);
    const uint32_t* rlast = nullptr;
    if constexpr (RS) {  // output row (b, limb) of [B][L]: input rows (b, limb) and (b, in_rows - 1)
        const size_t b = sg.row0 / a.L;
        rin = a.in + (b * a.in_rows + limb) * (size_t)N;
        rlast = a.in + (b * a.in_rows + a.in_rows - 1) * (size_t)N;
    }
    // the stages' twiddles are the same for every position: loaded once
    uint2 w[P - 1];
    load_tw_fwd<C::logP, LOGN, 0>(w, 0u, tw);
    // every input of every iteration is requested before the first is used (one DRAM round
    // trip; the cluster stores below are ordered memory operations the loads cannot pass)
    constexpr int PRE = RS ? 1 : ITERS;
    uint4 vin[PRE][P];
    if constexpr (PRE > 1) {
#pragma unroll
        for (int it = 0; it < ITERS; ++it) {
            const int j = (int)sg.part * share + (it * C::threads + (int)threadIdx.x) * 4;
#pragma unroll
            for (int t = 0; t < P; ++t) vin[it][t] = ld_had<F>(reinterpret_cast<const uint4*>(rin + j + t * C::m));
        }
    }
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int j = (int)sg.part * share + (it * C::threads + (int)threadIdx.x) * 4;
        uint4 v[P];
        if constexpr (PRE == 1) {
#pragma unroll
            for (int t = 0; t < P; ++t) v[t] = __ldg(reinterpret_cast<const uint4*>(rin + j + t * C::m));
        }
        if constexpr (RS) {
#pragma unroll
            for (int t = 0; t < P; ++t) {
                const uint4 wl = __ldg(reinterpret_cast<const uint4*>(rlast + j + t * C::m));
                v[t] = make_uint4(rescale_one(v[t].x, wl.x, lc), rescale_one(v[t].y, wl.y, lc),
                                  rescale_one(v[t].z, wl.z, lc), rescale_one(v[t].w, wl.w, lc));
            }
        }
        if constexpr (PRE > 1) {
#pragma unroll
            for (int t = 0; t < P; ++t) v[t] = vin[it][t];
        }
        uint32_t x[4][P];
#pragma unroll
        for (int t = 0; t < P; ++t) {
            x[0][t] = v[t].x;
            x[1][t] = v[t].y;
            x[2][t] = v[t].z;
            x[3][t] = v[t].w;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) fwd_stages_w<C::logP, LOGN, 0, F>(x[c], w, lc);
#pragma unroll
        for (int t = 0; t < P; ++t) st_cluster4(dst[t] + 4u * swz(j), make_uint4(x[0][t], x[1][t], x[2][t], x[3][t]));
    }
    cg::this_cluster().sync();
}

// Inverse stages LOGN-logP .. LOGN-1 of a split row (the scale N^-1, or N^-1 2^32, folded
// into the last): position j' < N/P is owned by one thread of the cluster (four consecutive
// positions per thread), which reads it from the P CTAs' shared memory and writes the P
// outputs j' + t N/P to global memory.  The closing barrier keeps this CTA's shared memory
// alive until its peers have read it.
template <int LOGN, int SCALE, int F>
__device__ __forceinline__ void inv_cross_pass(uint32_t* sm, const Seg& sg, const KArgs& a) {
    using C = Cfg<LOGN, F>;
    constexpr int N = 1 << LOGN, P = C::P, share = C::m / P, ITERS = share / (4 * C::threads);
    static_assert(share % (4 * C::threads) == 0, "whole uint4 groups per thread");
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();
    uint32_t src[P];
#pragma unroll
    for (int t = 0; t < P; ++t) src[t] = cluster_addr(sm, sg.rbase + t);
    const LimbConst& lc = row_lc<F>(a, sg.row0);
    const uint2* tw = row_twi<N, F>(a, sg.row0);
    uint32_t* out = row_out<N, F>(a, sg.row0);
    // twiddles shared by every position, and every peer read of every iteration, first
    uint2 w[P - 1];
    load_tw_inv<C::logP, LOGN, SCALE, LOGN - C::logP>(w, 0u, 0, tw);
    uint4 vin[ITERS][P];
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int j = (int)sg.part * share + (it * C::threads + (int)threadIdx.x) * 4;
#pragma unroll
        for (int t = 0; t < P; ++t) vin[it][t] = ld_cluster4(src[t] + 4u * swz(j));
    }
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int j = (int)sg.part * share + (it * C::threads + (int)threadIdx.x) * 4;
        uint32_t x[4][P];
#pragma unroll
        for (int t = 0; t < P; ++t) {
            x[0][t] = vin[it][t].x;
            x[1][t] = vin[it][t].y;
            x[2][t] = vin[it][t].z;
            x[3][t] = vin[it][t].w;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) inv_stages_w<C::logP, LOGN, SCALE, LOGN - C::logP, F>(x[c], w, lc);
#pragma unroll
        for (int t = 0; t < P; ++t)
            *reinterpret_cast<uint4*>(out + j + t * C::m) = make_uint4(x[0][t], x[1][t], x[2][t], x[3][t]);
    }
    cluster.sync();
}

// The inverse transforms of the contiguous layout take their input part by TMA (an async
// bulk copy into the swizzled shared layout, which is the tensor map's 128-byte swizzle);
// row lists (per-row pointers) and the Hadamard form keep the register loads.
template <int LOGN, int MODE, int F>
__host__ __device__ constexpr bool tma_input() {
    return MODE == MODE_INV && (F & 1) == 0 && LOGN >= 13;  // whole 256-line boxes per CTA
}
// The forward transforms of the contiguous layout write their part by TMA (the last pass
// reduces into the swizzled buffer, one thread stores it as 256-line boxes).
template <int LOGN, int MODE, int F>
__host__ __device__ constexpr bool tma_output() {
    return (MODE == MODE_FWD || MODE == MODE_RS_FWD) && (F & 1) == 0 && LOGN >= 13;
}
template <int LOGN, int MODE, int F>
__host__ __device__ constexpr bool uses_tma() {
    return tma_input<LOGN, MODE, F>() || tma_output<LOGN, MODE, F>();
}

// Where TMA does not apply (row lists, N < 2^13) the first inverse pass and the last forward
// pass still move whole lines: the CTA copies its rows between global and shared memory with
// lane-consecutive 16-byte accesses (the Hadamard product, if any, applied on the way in).
template <int LOGN, int F, bool HAD>
__device__ __forceinline__ void copy_in(uint32_t* sm, const Seg& sg, const KArgs& a) {
    using C = Cfg<LOGN, F>;
    constexpr int N = 1 << LOGN;
    for (int idx = threadIdx.x * 4; idx < sg.nrows * C::m; idx += C::threads * 4) {
        const int row = idx >> C::logm, i = idx & (C::m - 1);
        uint4 v = ld_had<F>(reinterpret_cast<const uint4*>(row_in<N, F>(a, sg.row0 + row) + sg.gbase + i));
        if constexpr (HAD) {
            const uint4 h = ld_had<F>(reinterpret_cast<const uint4*>(row_had<N, F>(a, sg.row0 + row) + sg.gbase + i));
            const LimbConst& lc = row_lc<F>(a, sg.row0 + row);
            v = make_uint4(mul_mont_lazy(v.x, h.x, lc.q, lc.qinv_neg), mul_mont_lazy(v.y, h.y, lc.q, lc.qinv_neg),
                           mul_mont_lazy(v.z, h.z, lc.q, lc.qinv_neg), mul_mont_lazy(v.w, h.w, lc.q, lc.qinv_neg));
        }
        *reinterpret_cast<uint4*>(&sm[swz(row * C::m + i)]) = v;
    }
    __syncthreads();
}

template <int LOGN, int F>
__device__ __forceinline__ void copy_out(const uint32_t* sm, const Seg& sg, const KArgs& a) {
    using C = Cfg<LOGN, F>;
    constexpr int N = 1 << LOGN;
    __syncthreads();
    for (int idx = threadIdx.x * 4; idx < sg.nrows * C::m; idx += C::threads * 4) {
        const int row = idx >> C::logm, i = idx & (C::m - 1);
        *reinterpret_cast<uint4*>(row_out<N, F>(a, sg.row0 + row) + sg.gbase + i) =
            *reinterpret_cast<const uint4*>(&sm[swz(row * C::m + i)]);
    }
}

// Stores the CTA's elems words (the buffer, swizzled) to the output by TMA and waits until
// the copy has read shared memory, so that the buffer may be reused or released.
template <int LOGN>
__device__ __forceinline__ void store_part_tma(uint32_t* sm, const Seg& sg, const KArgs& a) {
    using C = Cfg<LOGN>;
    constexpr int N = 1 << LOGN;
    constexpr int BOXES = C::elems / 8192;
    tc::fence_proxy_async_smem();  // this thread's buffer writes before the async-proxy read
    __syncthreads();
    if (threadIdx.x == 0) {
        const int32_t y0 = (int32_t)(((size_t)sg.row0 * N + sg.gbase) / 32);
#pragma unroll
        for (int b = 0; b < BOXES; ++b) tc::tma_store_2d(&a.tmap_out, 0, y0 + b * 256, sm + b * 8192);
        tc::bulk_commit();
        tc::bulk_wait_read0();
    }
    __syncthreads();
}

constexpr uint32_t kErrCcTma = 16;  // error code: the input copy did not arrive in time

// Copies the CTA's elems words (rows of 32 in 256-row boxes) into shared memory and waits
// (bounded) for them.  On a timeout the error flag is set and the task runs on to its end on
// whatever the buffer holds, so that every barrier is still reached.
template <int LOGN>
__device__ __forceinline__ void load_part_tma(uint32_t* sm, const Seg& sg, const KArgs& a, uint64_t* bar,
                                              uint32_t& phase) {
    using C = Cfg<LOGN>;
    constexpr int N = 1 << LOGN;
    constexpr int BOXES = C::elems / 8192;  // 256 rows of 32 words per box
    if (threadIdx.x == 0) {
        tc::fence_proxy_async_smem();  // earlier generic accesses of the buffer before the copy
        tc::mbar_arrive_expect_tx(bar, (uint32_t)C::elems * 4u);
        const int32_t y0 = (int32_t)(((size_t)sg.row0 * N + sg.gbase) / 32);
#pragma unroll
        for (int b = 0; b < BOXES; ++b) tc::tma_load_2d(sm + b * 8192, &a.tmap_in, 0, y0 + b * 256, bar);
    }
    tc::mbar_wait(bar, phase, a.err, kErrCcTma);
    phase ^= 1u;
}

template <int LOGN, int MODE, int F>
__device__ __forceinline__ void run_task(uint32_t* sm, const Seg& sg, const KArgs& a, uint64_t* tma_bar,
                                         uint32_t& tma_phase) {
    using C = Cfg<LOGN, F>;
    constexpr int RS = C::r_small;
    constexpr int S_FIRST = C::logP;              // first stage run inside the CTA
    constexpr int S_SMALL = LOGN - RS;            // first stage of the smallest-stride pass
    constexpr int FW = F | (((HEFX_CC_WIDE_MODES >> MODE) & 1) ? kWide : 0);  // F of the big-stride passes

    if constexpr (MODE == MODE_FWD || MODE == MODE_RS_FWD) {
        constexpr bool TMA = tma_output<LOGN, MODE, F>();
        static_assert(MODE == MODE_FWD || C::split, "the rescaling load is the cross-CTA pass");
        if constexpr (C::split) fwd_cross_pass<LOGN, F, MODE == MODE_RS_FWD>(sm, sg, a);
        if constexpr (C::nrest == 0) {
            static_assert(!TMA, "TMA output needs the smallest-stride pass to follow a shared-memory pass");
            fwd_pass<RS, LOGN, S_FIRST, C::split ? SRC_SMEM : SRC_GLOBAL, DST_GLOBAL_REDUCE, F>(sm, sg, a);
        } else {
            fwd_big<LOGN, 0, S_FIRST, FW>(sm, sg, a);
            fwd_pass<RS, LOGN, S_SMALL, SRC_SMEM, DST_SMEM_REDUCE, F>(sm, sg, a);
            if constexpr (TMA) store_part_tma<LOGN>(sm, sg, a);
            else copy_out<LOGN, F>(sm, sg, a);
        }
    } else if constexpr (MODE == MODE_INV || MODE == MODE_HAD_INV) {
        constexpr int SCALE = MODE == MODE_INV ? 1 : 2;
        constexpr bool TMA = tma_input<LOGN, MODE, F>();
        if constexpr (C::nrest == 0 && !C::split) {
            inv_pass<RS, LOGN, SCALE, 0, MODE == MODE_INV ? SRC_GLOBAL : SRC_GLOBAL_HAD, DST_GLOBAL, F>(sm, sg, a);
        } else {
            constexpr int SRC = SRC_SMEM;
            if constexpr (TMA) load_part_tma<LOGN>(sm, sg, a, tma_bar, tma_phase);
            else copy_in<LOGN, F, MODE == MODE_HAD_INV>(sm, sg, a);
            inv_pass<RS, LOGN, C::split ? 0 : SCALE, 0, SRC, DST_SMEM, F>(sm, sg, a);
            __syncthreads();
            inv_big<LOGN, SCALE, C::nrest - 1, RS, FW>(sm, sg, a);
            if constexpr (C::split) inv_cross_pass<LOGN, SCALE, F>(sm, sg, a);
        }
    } else {  // MODE_FWD_HAD_INV
        if constexpr (C::nrest == 0 && !C::split) {
            fwd_had_inv_pass<RS, LOGN, S_SMALL, SRC_GLOBAL, DST_GLOBAL, F>(sm, sg, a);
        } else {
            if constexpr (C::split) fwd_cross_pass<LOGN, F>(sm, sg, a);
            fwd_big<LOGN, 0, S_FIRST, FW>(sm, sg, a);
            fwd_had_inv_pass<RS, LOGN, S_SMALL, SRC_SMEM, DST_SMEM, F>(sm, sg, a);
            __syncthreads();
            inv_big<LOGN, 2, C::nrest - 1, RS, FW>(sm, sg, a);
            if constexpr (C::split) inv_cross_pass<LOGN, 2, F>(sm, sg, a);
        }
    }
}

template <int LOGN, int MODE, int F>
__global__ void __launch_bounds__(Cfg<LOGN, F>::threads, Cfg<LOGN, F>::minb) ntt_cc_kernel(const __grid_constant__ KArgs a) {
    using C = Cfg<LOGN, F>;
    extern __shared__ __align__(16) uint32_t sm_raw[];
    __shared__ uint64_t tma_bar;
    uint32_t tma_phase = 0;
    uint32_t* sm = sm_raw;
    if constexpr (uses_tma<LOGN, MODE, F>()) {
        // the 128-byte swizzle repeats every 1024 bytes: align the buffer to it (1 KiB extra)
        const uint32_t s0 = tc::smem_u32(sm_raw);
        sm = sm_raw + ((((s0 + 1023u) & ~1023u) - s0) >> 2);
        if (threadIdx.x == 0) {
            tc::mbar_init(&tma_bar, 1);
            tc::fence_mbar_init();
        }
        __syncthreads();
    }
    // programmatic dependent launch: every global access (and every cluster access) is below
    griddep_wait();
    // persistent: each CTA (or cluster of P CTAs) walks a strided sequence of tasks; a task
    // is one row (split N) or C::rows rows
    const uint32_t ntasks = C::split ? a.rows : (a.rows + C::rows - 1) / C::rows;
    const uint32_t first = blockIdx.x >> C::logP;
    const uint32_t stride = gridDim.x >> C::logP;
    for (uint32_t task = first; task < ntasks; task += stride) {
        Seg sg;
        if constexpr (C::split) {
            sg.row0 = task;
            sg.part = blockIdx.x & (C::P - 1);  // == rank in the cluster
            sg.nrows = 1;
        } else {
            sg.row0 = task * C::rows;
            sg.part = 0;
            sg.nrows = (int)min((uint32_t)C::rows, a.rows - sg.row0);
        }
        sg.gbase = sg.part * C::m;
        sg.rbase = 0;
        run_task<LOGN, MODE, F>(sm, sg, a, &tma_bar, tma_phase);
        // shared memory is reused by the next task; with a split row the peers write into it
        if (task + stride < ntasks) sync_all<C::split>();
    }
}

// rows == 0: set the kernel's attributes only (done before a stream capture).
template <int LOGN, int MODE, int F>
cudaError_t launch_one(const KArgs& a, size_t rows, cudaStream_t stream) {
    using C = Cfg<LOGN, F>;
    auto kern = ntt_cc_kernel<LOGN, MODE, F>;
    constexpr int smem = C::smem_bytes + (uses_tma<LOGN, MODE, F>() ? 1024 : 0);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    cfg.blockDim = dim3(C::threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    // the set-up may overlap the stream's preceding kernel; the kernel waits (griddep_wait)
    // before its first memory access
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (C::split) {
        attr[1].id = cudaLaunchAttributeClusterDimension;
        attr[1].val.clusterDim.x = C::P;
        attr[1].val.clusterDim.y = 1;
        attr[1].val.clusterDim.z = 1;
        cfg.numAttrs = 2;
    }
    // One CTA (cluster) per task, scheduled by the hardware: measured faster than persistent
    // grids, both with an equal number of tasks per CTA (whose lower occupancy costs more
    // than a partial last wave) and walking row lists from the co-resident count (config-4
    // batch 1.30 vs 1.35 ms).  The kernel still loops, so a smaller grid would stay correct.
    int dev = 0;
    cudaGetDevice(&dev);
    static bool attr_set[64] = {};  // per template instance and device; benign race (idempotent)
    if (!attr_set[dev & 63]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set[dev & 63] = true;
    }
    if (rows == 0) return cudaSuccess;
    const size_t groups = C::split ? rows : (rows + C::rows - 1) / C::rows;
    cfg.gridDim = dim3((unsigned)(C::P * groups));
    return cudaLaunchKernelEx(&cfg, kern, a);
}

// Clusters of this kernel configuration that fit on the device at once (the occupancy the
// runtime reports), 0 for unsplit rows or where it cannot be queried.
template <int LOGN, int MODE, int F>
int max_active_clusters() {
    using C = Cfg<LOGN, F>;
    if constexpr (!C::split) {
        return 0;
    } else {
        KArgs dummy = {};
        if (launch_one<LOGN, MODE, F>(dummy, 0, nullptr) != cudaSuccess) return 0;  // sets the smem attribute
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        cfg.gridDim = dim3((unsigned)(C::P * 1024));
        cfg.blockDim = dim3(C::threads);
        cfg.dynamicSmemBytes = C::smem_bytes + (uses_tma<LOGN, MODE, F>() ? 1024 : 0);
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C::P;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, ntt_cc_kernel<LOGN, MODE, F>, &cfg) != cudaSuccess) return 0;
        return n;
    }
}

template <int LOGN, int F>
cudaError_t launch_mode_d(NttMode mode, const KArgs& a, size_t rows, cudaStream_t s) {
    switch (mode) {
        case MODE_FWD: return launch_one<LOGN, MODE_FWD, F>(a, rows, s);
        case MODE_INV: return launch_one<LOGN, MODE_INV, F>(a, rows, s);
        case MODE_FWD_HAD_INV: return launch_one<LOGN, MODE_FWD_HAD_INV, F>(a, rows, s);
        case MODE_RS_FWD:
            if constexpr ((F & 1) == 0 && Cfg<LOGN>::split) return launch_one<LOGN, MODE_RS_FWD, F>(a, rows, s);
            else return cudaErrorNotSupported;
        default: return launch_one<LOGN, MODE_HAD_INV, F>(a, rows, s);
    }
}

// lazy: every modulus of the parameter set is below 2^28
template <int LOGN>
cudaError_t launch_mode(NttMode mode, const KArgs& a, size_t rows, cudaStream_t s, bool lazy) {
    if (a.desc) return lazy ? launch_mode_d<LOGN, 3>(mode, a, rows, s) : launch_mode_d<LOGN, 1>(mode, a, rows, s);
    return lazy ? launch_mode_d<LOGN, 2>(mode, a, rows, s) : launch_mode_d<LOGN, 0>(mode, a, rows, s);
}

// Co-resident clusters of the contiguous-layout forward or inverse kernel at N = 2^16
// (ntt_cc_range_d.cu), 0 where it cannot be queried.
int max_clusters_16(NttMode mode, bool lazy);

// One LOGN range of the dispatcher, compiled in its own translation unit (build time).
cudaError_t launch_range_a(int logn, NttMode mode, const KArgs& a, size_t rows, cudaStream_t s, bool lazy);
cudaError_t launch_range_b(int logn, NttMode mode, const KArgs& a, size_t rows, cudaStream_t s, bool lazy);
cudaError_t launch_range_c(int logn, NttMode mode, const KArgs& a, size_t rows, cudaStream_t s, bool lazy);
cudaError_t launch_range_d(int logn, NttMode mode, const KArgs& a, size_t rows, cudaStream_t s, bool lazy);
cudaError_t launch_range_e(int logn, NttMode mode, const KArgs& a, size_t rows, cudaStream_t s, bool lazy);

}  // namespace cc
}  // namespace hefx
