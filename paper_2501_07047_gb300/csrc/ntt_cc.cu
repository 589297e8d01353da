// CUDA-core negacyclic NTT / INTT (path a): radix-2 Cooley-Tukey forward and
// Gentleman-Sande inverse (App. A, "Radix-2 Cooley-Tukey NTT"; the garbled loop indices of
// the printed algorithm are replaced by the textbook ones), with lazy Shoup butterflies.
//
// GB300 mapping
//  - One CTA holds a whole limb (N <= 2^15) or half of one (N = 2^16) in shared memory,
//    so each limb is read from and written to HBM once per transform (512 KiB per
//    N = 2^16 limb-NTT).  A CTA with N < 2^13 holds 2^13 / N limbs.
//  - N = 2^16 uses a 2-CTA cluster.  Forward: the first stage (pairs j, j + N/2) is
//    computed while loading, each CTA producing its own half (both read the whole limb,
//    the second read hits L2).  Inverse: the last stage is exchanged through distributed
//    shared memory.
//  - Stages run in register passes of up to 5 stages (radix-32 sub-transforms); each pass
//    reads and writes shared memory once.  Shared memory is padded by one word per 32 so
//    that both strided and contiguous sub-transform accesses are bank-conflict free.
//  - The forward output is in bit-reversed order with no shuffle (the twiddle table is
//    stored in bit-reversed order, as MAT folds permutations into constants, Sec. IV-B).
#include <cooperative_groups.h>

#include "hefx_internal.h"
#include "modarith.cuh"

namespace cg = cooperative_groups;

namespace hefx {
namespace {

__device__ __forceinline__ int pad(int j) { return j + (j >> 5); }

template <int LOGN>
struct Cfg {
    static constexpr bool split = LOGN >= 16;
    static constexpr int logm = split ? LOGN - 1 : LOGN;  // elements of one row segment
    static constexpr int m = 1 << logm;
    static constexpr int rows = logm >= 13 ? 1 : (1 << (13 - logm));  // row segments per CTA
    static constexpr int elems = m * rows;
    static constexpr int threads = elems >= (1 << 14) ? 512 : 256;
    static constexpr int smem_bytes = (elems + elems / 32) * 4;
    static constexpr int S = logm;                  // stages run inside the CTA
    static constexpr int r_small = S < 5 ? S : 5;   // pass over the smallest strides
    static constexpr int rest = S - r_small;
    static constexpr int nrest = (rest + 4) / 5;
    __host__ __device__ static constexpr int big(int i) {
        return nrest == 0 ? 0 : rest / nrest + (i < rest % nrest ? 1 : 0);
    }
};

struct KArgs {
    const uint32_t* in;
    const uint32_t* had;
    uint32_t* out;
    const uint2* tw_f;  // forward twiddles [L][N]
    const uint2* tw_i;  // inverse twiddles [L][N]
    const LimbConst* lc;
    uint32_t rows;
    uint32_t L;
};

// Forward pass over global stages s0 .. s0+R-1 (stage s pairs j, j + N/2^(s+1)).
template <int R, int LOGN, int s0>
__device__ __forceinline__ void fwd_pass(uint32_t* sm, uint32_t gbase, uint32_t row0, const KArgs& a) {
    using C = Cfg<LOGN>;
    constexpr int N = 1 << LOGN;
    constexpr int logtl = LOGN - s0 - R;  // log2 of the smallest stride of the pass
    constexpr int lognsub = C::logm - R;
    constexpr int nsub = 1 << lognsub;
    for (int u = threadIdx.x; u < C::rows * nsub; u += C::threads) {
        const int row = u >> lognsub;
        const int uu = u & (nsub - 1);
        const int j_lo = uu & ((1 << logtl) - 1);
        const int j_hi = uu >> logtl;
        const int jb = row * C::m + (j_hi << (logtl + R)) + j_lo;
        const uint32_t g0 = (gbase >> (logtl + R)) + (uint32_t)j_hi;
        const uint32_t limb = (row0 + row) % a.L;
        const uint32_t q = a.lc[limb].q;
        const uint2* tw = a.tw_f + (size_t)limb * N;
        uint32_t x[1 << R];
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) x[k] = sm[pad(jb + (k << logtl))];
        // constant trip counts at every loop level so that full unrolling keeps x[] in registers
#pragma unroll
        for (int v = 0; v < R; ++v) {
#pragma unroll
            for (int b = 0; b < (1 << (R - 1)); ++b) {
                const int half = 1 << (R - 1 - v);
                const int g = b >> (R - 1 - v);
                const int k = (g << (R - v)) + (b & (half - 1));
                const uint2 w = __ldg(&tw[(1u << (s0 + v)) + (g0 << v) + g]);
                ct_bfly(x[k], x[k + half], w.x, w.y, q);
            }
        }
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) sm[pad(jb + (k << logtl))] = x[k];
    }
}

// Inverse pass over Gentleman-Sande stages e0 .. e0+R-1 (stage e pairs j, j + 2^e).
// SCALE selects the N^-1 factor folded into the last stage of the whole transform
// (0: none, 1: N^-1, 2: N^-1 * 2^32 after a Montgomery Hadamard product).
template <int R, int LOGN, int SCALE, int e0>
__device__ __forceinline__ void inv_pass(uint32_t* sm, uint32_t gbase, uint32_t row0, const KArgs& a) {
    using C = Cfg<LOGN>;
    constexpr int N = 1 << LOGN;
    constexpr int lognsub = C::logm - R;
    constexpr int nsub = 1 << lognsub;
    for (int u = threadIdx.x; u < C::rows * nsub; u += C::threads) {
        const int row = u >> lognsub;
        const int uu = u & (nsub - 1);
        const int j_lo = uu & ((1 << e0) - 1);
        const int j_hi = uu >> e0;
        const int jb = row * C::m + (j_hi << (e0 + R)) + j_lo;
        const uint32_t limb = (row0 + row) % a.L;
        const LimbConst& lc = a.lc[limb];
        const uint32_t q = lc.q;
        const uint2* tw = a.tw_i + (size_t)limb * N;
        uint32_t x[1 << R];
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) x[k] = sm[pad(jb + (k << e0))];
#pragma unroll
        for (int v = 0; v < R; ++v) {
            const int e = e0 + v;
            const int h = 1 << v;
            if (SCALE && e == LOGN - 1) {
                // last stage of the transform: one group, twiddle psi^-brv(1), times N^-1
                const uint32_t s = SCALE == 1 ? lc.ninv : lc.ninvR, ssh = SCALE == 1 ? lc.ninv_sh : lc.ninvR_sh;
                const uint32_t w = SCALE == 1 ? lc.ninvw : lc.ninvRw, wsh = SCALE == 1 ? lc.ninvw_sh : lc.ninvRw_sh;
#pragma unroll
                for (int kk = 0; kk < (1 << (R - 1)); ++kk) {
                    const uint32_t X = x[kk], Y = x[kk + h];
                    x[kk] = csub(mul_shoup_lazy(X + Y, s, ssh, q), q);
                    x[kk + h] = csub(mul_shoup_lazy(X - Y + 2 * q, w, wsh, q), q);
                }
                continue;
            }
            const uint32_t hbase = (uint32_t)(N >> (e + 1)) + (gbase >> (e + 1)) + ((uint32_t)j_hi << (R - v - 1));
#pragma unroll
            for (int b = 0; b < (1 << (R - 1)); ++b) {
                const int g = b >> v;
                const int k = (g << (v + 1)) + (b & (h - 1));
                const uint2 w = __ldg(&tw[hbase + g]);
                gs_bfly(x[k], x[k + h], w.x, w.y, q);
            }
        }
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) sm[pad(jb + (k << e0))] = x[k];
    }
}

template <int LOGN, int I, int s>
__device__ __forceinline__ void run_fwd_from(uint32_t* sm, uint32_t gbase, uint32_t row0, const KArgs& a) {
    using C = Cfg<LOGN>;
    if constexpr (I < C::nrest) {
        constexpr int r = C::big(I);
        fwd_pass<r, LOGN, s>(sm, gbase, row0, a);
        __syncthreads();
        run_fwd_from<LOGN, I + 1, s + r>(sm, gbase, row0, a);
    } else {
        fwd_pass<C::r_small, LOGN, s>(sm, gbase, row0, a);
        __syncthreads();
    }
}

template <int LOGN>
__device__ __forceinline__ void run_fwd(uint32_t* sm, uint32_t gbase, uint32_t row0, const KArgs& a) {
    run_fwd_from<LOGN, 0, Cfg<LOGN>::split ? 1 : 0>(sm, gbase, row0, a);
}

template <int LOGN, int SCALE, int I, int e>
__device__ __forceinline__ void run_inv_from(uint32_t* sm, uint32_t gbase, uint32_t row0, const KArgs& a) {
    using C = Cfg<LOGN>;
    if constexpr (I >= 0) {
        constexpr int r = C::big(I);
        inv_pass<r, LOGN, SCALE, e>(sm, gbase, row0, a);
        __syncthreads();
        run_inv_from<LOGN, SCALE, I - 1, e + r>(sm, gbase, row0, a);
    }
}

template <int LOGN, int SCALE>
__device__ __forceinline__ void run_inv(uint32_t* sm, uint32_t gbase, uint32_t row0, const KArgs& a) {
    using C = Cfg<LOGN>;
    inv_pass<C::r_small, LOGN, SCALE, 0>(sm, gbase, row0, a);
    __syncthreads();
    run_inv_from<LOGN, SCALE, C::nrest - 1, C::r_small>(sm, gbase, row0, a);
}

template <int LOGN, int MODE>
__global__ void __launch_bounds__(Cfg<LOGN>::threads) ntt_cc_kernel(KArgs a) {
    using C = Cfg<LOGN>;
    constexpr int N = 1 << LOGN;
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t row0, half = 0;
    if (C::split) {
        row0 = blockIdx.x >> 1;
        half = blockIdx.x & 1;
    } else {
        row0 = blockIdx.x * C::rows;
    }
    const uint32_t gbase = half * C::m;
    const int nrows = C::split ? 1 : (int)min((uint32_t)C::rows, a.rows - row0);

    // ---- copy-in (coalesced, 4 consecutive words per thread)
    for (int i = threadIdx.x * 4; i < C::elems; i += C::threads * 4) {
        const int row = i >> C::logm;
        const int j = i & (C::m - 1);
        uint4 v = make_uint4(0, 0, 0, 0);
        if (row < nrows) {
            const size_t g = (size_t)(row0 + row) * N + gbase + j;
            const uint32_t limb = (row0 + row) % a.L;
            const LimbConst& lc = a.lc[limb];
            if (C::split && (MODE == MODE_FWD || MODE == MODE_FWD_HAD_INV)) {
                // first forward stage fused: X + w Y (half 0) or X - w Y (half 1), w = psi^brv(1)
                const size_t g0 = (size_t)(row0 + row) * N + j;
                const uint4 X = *reinterpret_cast<const uint4*>(a.in + g0);
                const uint4 Y = *reinterpret_cast<const uint4*>(a.in + g0 + N / 2);
                const uint2 w = __ldg(&a.tw_f[(size_t)limb * N + 1]);
                const uint32_t q = lc.q;
                uint32_t xs[4] = {X.x, X.y, X.z, X.w}, ys[4] = {Y.x, Y.y, Y.z, Y.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint32_t tt = mul_shoup_lazy(ys[t], w.x, w.y, q);
                    xs[t] = half ? xs[t] - tt + 2 * q : xs[t] + tt;
                }
                v = make_uint4(xs[0], xs[1], xs[2], xs[3]);
            } else {
                v = *reinterpret_cast<const uint4*>(a.in + g);
                if (MODE == MODE_HAD_INV) {
                    const uint4 h = *reinterpret_cast<const uint4*>(a.had + g);
                    v.x = mul_mont_lazy(v.x, h.x, lc.q, lc.qinv_neg);
                    v.y = mul_mont_lazy(v.y, h.y, lc.q, lc.qinv_neg);
                    v.z = mul_mont_lazy(v.z, h.z, lc.q, lc.qinv_neg);
                    v.w = mul_mont_lazy(v.w, h.w, lc.q, lc.qinv_neg);
                }
            }
        }
        sm[pad(i)] = v.x;
        sm[pad(i + 1)] = v.y;
        sm[pad(i + 2)] = v.z;
        sm[pad(i + 3)] = v.w;
    }
    if (C::split) {
        cg::this_cluster().sync();  // both CTAs finished reading before anyone writes (in-place safety)
    } else {
        __syncthreads();
    }

    if (MODE == MODE_FWD || MODE == MODE_FWD_HAD_INV) run_fwd<LOGN>(sm, gbase, row0, a);

    if (MODE == MODE_FWD_HAD_INV) {
        for (int i = threadIdx.x; i < C::elems; i += C::threads) {
            const int row = i >> C::logm;
            if (row < nrows) {
                const LimbConst& lc = a.lc[(row0 + row) % a.L];
                const uint32_t h = a.had[(size_t)(row0 + row) * N + gbase + (i & (C::m - 1))];
                sm[pad(i)] = mul_mont_lazy(sm[pad(i)], h, lc.q, lc.qinv_neg);
            }
        }
        __syncthreads();
    }

    if (MODE == MODE_FWD) {
        for (int i = threadIdx.x * 4; i < C::elems; i += C::threads * 4) {
            const int row = i >> C::logm;
            if (row >= nrows) continue;
            const uint32_t q = a.lc[(row0 + row) % a.L].q;
            uint4 v;
            v.x = reduce4(sm[pad(i)], q);
            v.y = reduce4(sm[pad(i + 1)], q);
            v.z = reduce4(sm[pad(i + 2)], q);
            v.w = reduce4(sm[pad(i + 3)], q);
            *reinterpret_cast<uint4*>(a.out + (size_t)(row0 + row) * N + gbase + (i & (C::m - 1))) = v;
        }
        return;
    }

    constexpr int SCALE = (MODE == MODE_INV) ? 1 : 2;
    if (!C::split) {
        run_inv<LOGN, SCALE>(sm, gbase, row0, a);
        for (int i = threadIdx.x * 4; i < C::elems; i += C::threads * 4) {
            const int row = i >> C::logm;
            if (row >= nrows) continue;
            const uint4 v = make_uint4(sm[pad(i)], sm[pad(i + 1)], sm[pad(i + 2)], sm[pad(i + 3)]);
            *reinterpret_cast<uint4*>(a.out + (size_t)(row0 + row) * N + gbase + (i & (C::m - 1))) = v;
        }
        return;
    }

    // split inverse: stages with stride < N/2 are local; the last one pairs the two halves
    run_inv<LOGN, 0>(sm, gbase, row0, a);
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();
    {
        const uint32_t* s0 = cluster.map_shared_rank(sm, 0);
        const uint32_t* s1 = cluster.map_shared_rank(sm, 1);
        const LimbConst& lc = a.lc[row0 % a.L];
        const uint32_t q = lc.q;
        const uint32_t s = SCALE == 1 ? lc.ninv : lc.ninvR, ssh = SCALE == 1 ? lc.ninv_sh : lc.ninvR_sh;
        const uint32_t w = SCALE == 1 ? lc.ninvw : lc.ninvRw, wsh = SCALE == 1 ? lc.ninvw_sh : lc.ninvRw_sh;
        uint32_t* out = a.out + (size_t)row0 * N;
        for (int i = threadIdx.x * 4; i < N / 4; i += C::threads * 4) {
            const int j = half * (N / 4) + i;
            uint32_t r0[4], r1[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint32_t X = s0[pad(j + t)], Y = s1[pad(j + t)];
                r0[t] = csub(mul_shoup_lazy(X + Y, s, ssh, q), q);
                r1[t] = csub(mul_shoup_lazy(X - Y + 2 * q, w, wsh, q), q);
            }
            *reinterpret_cast<uint4*>(out + j) = make_uint4(r0[0], r0[1], r0[2], r0[3]);
            *reinterpret_cast<uint4*>(out + j + N / 2) = make_uint4(r1[0], r1[1], r1[2], r1[3]);
        }
    }
    cluster.sync();  // keep this CTA's shared memory alive until the peer has read it
}

template <int LOGN, int MODE>
cudaError_t launch_one(const KArgs& a, size_t rows, cudaStream_t stream) {
    using C = Cfg<LOGN>;
    auto kern = ntt_cc_kernel<LOGN, MODE>;
    static bool attr_done = false;  // per template instance; benign race (idempotent call)
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::smem_bytes);
        if (e != cudaSuccess) return e;
        if (C::split) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
            (void)e;
        }
        attr_done = true;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(C::threads);
    cfg.dynamicSmemBytes = C::smem_bytes;
    cfg.stream = stream;
    if (C::split) {
        cfg.gridDim = dim3((unsigned)(rows * 2));
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    } else {
        cfg.gridDim = dim3((unsigned)((rows + C::rows - 1) / C::rows));
    }
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int LOGN>
cudaError_t launch_mode(NttMode mode, const KArgs& a, size_t rows, cudaStream_t s) {
    switch (mode) {
        case MODE_FWD: return launch_one<LOGN, MODE_FWD>(a, rows, s);
        case MODE_INV: return launch_one<LOGN, MODE_INV>(a, rows, s);
        case MODE_FWD_HAD_INV: return launch_one<LOGN, MODE_FWD_HAD_INV>(a, rows, s);
        default: return launch_one<LOGN, MODE_HAD_INV>(a, rows, s);
    }
}

}  // namespace

cudaError_t launch_ntt_cc(const hefx_params* p, NttMode mode, const uint32_t* in, const uint32_t* had, uint32_t* out,
                          size_t rows, cudaStream_t stream) {
    KArgs a;
    a.in = in;
    a.had = had;
    a.out = out;
    a.tw_f = p->d_tw_fwd;
    a.tw_i = p->d_tw_inv;
    a.lc = p->d_lc;
    a.rows = (uint32_t)rows;
    a.L = p->nlimbs;
    if (rows == 0) return cudaSuccess;
    switch (p->log2n) {
        case 3: return launch_mode<3>(mode, a, rows, stream);
        case 4: return launch_mode<4>(mode, a, rows, stream);
        case 5: return launch_mode<5>(mode, a, rows, stream);
        case 6: return launch_mode<6>(mode, a, rows, stream);
        case 7: return launch_mode<7>(mode, a, rows, stream);
        case 8: return launch_mode<8>(mode, a, rows, stream);
        case 9: return launch_mode<9>(mode, a, rows, stream);
        case 10: return launch_mode<10>(mode, a, rows, stream);
        case 11: return launch_mode<11>(mode, a, rows, stream);
        case 12: return launch_mode<12>(mode, a, rows, stream);
        case 13: return launch_mode<13>(mode, a, rows, stream);
        case 14: return launch_mode<14>(mode, a, rows, stream);
        case 15: return launch_mode<15>(mode, a, rows, stream);
        case 16: return launch_mode<16>(mode, a, rows, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hefx
