// CUDA-core negacyclic NTT / INTT of N = 2^16 rows in two passes through L2 (path a, the
// two-pass schedule of the contiguous [rows][N] transforms at this ring degree).
//
// The radix-2 Cooley-Tukey forward transform (App. A; the same butterflies, twiddles and lazy
// ranges as ntt_cc_impl.cuh) splits at stage 8: stages 0..7 pair elements j, j + 2^(15-s)
// whose indices agree mod 256 (a "column" j = c + 256 r of fixed c), and their twiddles depend
// on r only; stages 8..15 pair elements of one 256-element block (j >> 8 fixed).  This is the
// row / column factorisation of the matrix NTT (MAT, Sec. IV-B) with the twiddle step folded
// into the butterflies' own twiddles, so the two passes need no separate multiply:
//  - column pass: a CTA takes 16 columns x 256 r of one row (16 KiB); each thread runs a
//    radix-16 sub-transform over r = t + 16k, then (through shared memory, after a CTA
//    barrier) one over r = 16t + k;
//  - block pass: a CTA takes 16 blocks of 256 elements; each half-warp owns a block and runs a
//    radix-16 sub-transform over i = t + 16k, then (through the half-warp's shared memory, no
//    CTA barrier) one over i = 16t + k.
// The inverse (Gentleman-Sande) runs the same passes in the other order.  The intermediate
// goes through the output buffer (48 MiB for 192 rows stays resident in the 126 MB L2 between
// the two launches).  Against the single-launch cluster kernel this trades the cross-CTA step
// (distributed shared memory and two cluster barriers per row) for a second launch and many
// small CTAs: faster for small batches, whose rows are too few to fill the GPU with clusters
// (24 rows of 2^16: 16.9 / 15.4 us against 20.8 / 20.5 us), slower for large ones.  Global
// accesses move whole 32-byte sectors (16 consecutive words per half-warp); the
// smallest-stride pass reads its twiddles from the group-major table part (RS = 4 stages, laid
// out by hefx_params_create) so that lanes read consecutive entries.
#include "ntt_cc_impl.cuh"

namespace hefx {
namespace cc2 {

using cc::fwd_stages_w;
using cc::inv_stages_w;
using cc::load_tw_fwd;
using cc::load_tw_inv;
using cc::reduce_out;

constexpr int LOGN = 16, N = 1 << LOGN;
constexpr int THREADS = 256;  // 16 columns (or blocks) x 16 sub-transforms per CTA
constexpr int TASKS_PER_ROW = 16;

#ifndef HEFX_2P_MINB
#define HEFX_2P_MINB 4
#endif

struct Args2 {
    const uint32_t* in;
    uint32_t* out;
    const uint2* tw;  // [L][N]: the direction's table in the two-pass layout
    const LimbConst* lc;
    uint32_t L;
};

// Shared layout of a 256 x 16 column tile: element (r, c) at word 32 (r >> 1) + 16 h + c with
// h = bit 0 of r XOR bit 4 of r, so that both patterns (lanes over c for rows t, t + 1 and for
// rows 16t, 16t + 16) touch 32 different banks.  ColAddr holds, per thread (c, t), the two
// bases of each pattern (k even / odd); the per-k part is a compile-time offset.
struct ColAddr {
    int a[2], b[2];
    __device__ ColAddr(int c, int t) {
        a[0] = ((t >> 1) << 5) + ((t & 1) << 4) + c;  // r = t + 16k: + 256 k
        a[1] = ((t >> 1) << 5) + (((t & 1) ^ 1) << 4) + c;
        b[0] = (t << 8) + ((t & 1) << 4) + c;  // r = 16t + k: + 32 (k >> 1)
        b[1] = (t << 8) + (((t & 1) ^ 1) << 4) + c;
    }
    template <int k>
    __device__ int wa() const { return a[k & 1] + 256 * k; }
    template <int k>
    __device__ int wb() const { return b[k & 1] + 32 * (k >> 1); }
};

// Shared layout of a 16 x 256 block tile: element i of block bl at word 256 bl + swz(i ^ 16 h),
// h = bl & 1 (swz: the 16-byte-chunk XOR of ntt_cc_impl.cuh; the flip of bit 4 in odd blocks
// puts the two half-warps of a scalar access on different banks).  BlkAddr holds, per thread
// (bl, i), the bases of the scalar pattern (elements i + 16k) and of the uint4 pattern
// (elements 16i + 4q .. +3).
struct BlkAddr {
    int s[2][4];  // scalar: [parity of k ^ bit 3 of k][bits 1-2 of k]
    int v0, qx;   // uint4: word v0 + 4 (q ^ qx)
    __device__ BlkAddr(int bl, int i) {
        const int h16 = (bl & 1) << 4, base = bl << 8;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            s[0][j] = base + (i ^ (4 * j)) + h16;
            s[1][j] = base + (i ^ (4 * j)) - h16;
        }
        const int i1 = i ^ (bl & 1);  // 16 i ^ 16 h = 16 (i ^ h)
        v0 = base + ((16 * i1) ^ ((((i1 >> 1) & 7) << 2) & 16));
        qx = (i1 >> 1) & 3;
    }
    // swz(i + 16 k') with k' = k ^ h: (16 (k' ^ e)) + (i ^ 4 ((k >> 1) & 3)), e = bit 3 of k;
    // flipping bit 0 of k ^ e by h adds +16 h when it is even and -16 h when it is odd
    template <int k>
    __device__ int ws() const {
        constexpr int ke = k ^ ((k >> 3) & 1);
        return s[ke & 1][(k >> 1) & 3] + 16 * ke;
    }
    __device__ int wv(int q) const { return v0 + 4 * (q ^ qx); }
};

template <int K, class Fn>
__device__ __forceinline__ void unroll16(Fn&& f) {
    if constexpr (K < 16) {
        f(std::integral_constant<int, K>{});
        unroll16<K + 1>(f);
    }
}

// Forward stages 0..7 of 16 columns of one row: in -> out.
template <int F>
__global__ void __launch_bounds__(THREADS, HEFX_2P_MINB) fwd_cols_kernel(const Args2 a) {
    __shared__ uint32_t sm[16 * 256];
    griddep_wait();
    const uint32_t row = blockIdx.x / TASKS_PER_ROW;
    const uint32_t c0 = (blockIdx.x % TASKS_PER_ROW) * 16;
    const uint32_t limb = row % a.L;
    const LimbConst& lc = a.lc[limb];
    const uint2* tw = a.tw + (size_t)limb * N;
    const int c = threadIdx.x & 15, t = threadIdx.x >> 4;
    const ColAddr ad(c, t);
    const uint32_t* src = a.in + (size_t)row * N + c0 + c + 256 * t;
    uint32_t x[16];
    uint2 w[15];
    load_tw_fwd<4, LOGN, 0>(w, 0u, tw);
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = __ldcs(src + 4096 * k);
    fwd_stages_w<4, LOGN, 0, F>(x, w, lc);
    unroll16<0>([&](auto K) {
        constexpr int k = decltype(K)::value;
        sm[ad.wa<k>()] = x[k];
    });
    __syncthreads();  // every input of the tile is read before any output is written (in place)
    load_tw_fwd<4, LOGN, 4>(w, (uint32_t)t, tw);
    unroll16<0>([&](auto K) {
        constexpr int k = decltype(K)::value;
        x[k] = sm[ad.wb<k>()];
    });
    fwd_stages_w<4, LOGN, 4, F>(x, w, lc);
    uint32_t* dst = a.out + (size_t)row * N + c0 + c + 4096 * t;
#pragma unroll
    for (int k = 0; k < 16; ++k) dst[256 * k] = x[k];
}

// Forward stages 8..15 of 16 blocks of one row, in place in out; canonical outputs.
template <int F>
__global__ void __launch_bounds__(THREADS, HEFX_2P_MINB) fwd_rows_kernel(const Args2 a) {
    __shared__ __align__(16) uint32_t sm[16 * 256];
    griddep_wait();
    const uint32_t row = blockIdx.x / TASKS_PER_ROW;
    const uint32_t limb = row % a.L;
    const LimbConst& lc = a.lc[limb];
    const uint2* tw = a.tw + (size_t)limb * N;
    const int bl = threadIdx.x >> 4, i = threadIdx.x & 15;
    const uint32_t b = (blockIdx.x % TASKS_PER_ROW) * 16 + bl;  // block of the row
    const BlkAddr ad(bl, i);
    uint32_t* base = a.out + (size_t)row * N + (b << 8);
    uint32_t x[16];
    uint2 w[15];
    load_tw_fwd<4, LOGN, 8>(w, b, tw);
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = __ldcg(base + i + 16 * k);
    fwd_stages_w<4, LOGN, 8, F>(x, w, lc);
    unroll16<0>([&](auto K) {
        constexpr int k = decltype(K)::value;
        sm[ad.ws<k>()] = x[k];
    });
    __syncwarp();  // a block is exchanged within its half-warp
    load_tw_fwd<4, LOGN, 12>(w, (b << 4) + (uint32_t)i, tw);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 v = *reinterpret_cast<const uint4*>(&sm[ad.wv(q)]);
        x[4 * q] = v.x;
        x[4 * q + 1] = v.y;
        x[4 * q + 2] = v.z;
        x[4 * q + 3] = v.w;
    }
    fwd_stages_w<4, LOGN, 12, F>(x, w, lc);
    uint4* dst = reinterpret_cast<uint4*>(base + 16 * i);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        dst[q] = make_uint4(reduce_out<F>(x[4 * q], lc), reduce_out<F>(x[4 * q + 1], lc),
                            reduce_out<F>(x[4 * q + 2], lc), reduce_out<F>(x[4 * q + 3], lc));
}

// Inverse stages 0..7 of 16 blocks of one row: in -> out.
template <int F>
__global__ void __launch_bounds__(THREADS, HEFX_2P_MINB) inv_rows_kernel(const Args2 a) {
    __shared__ __align__(16) uint32_t sm[16 * 256];
    griddep_wait();
    const uint32_t row = blockIdx.x / TASKS_PER_ROW;
    const uint32_t limb = row % a.L;
    const LimbConst& lc = a.lc[limb];
    const uint2* tw = a.tw + (size_t)limb * N;
    const int bl = threadIdx.x >> 4, i = threadIdx.x & 15;
    const uint32_t b = (blockIdx.x % TASKS_PER_ROW) * 16 + bl;
    const BlkAddr ad(bl, i);
    const uint4* src = reinterpret_cast<const uint4*>(a.in + (size_t)row * N + (b << 8) + 16 * i);
    uint32_t x[16];
    uint2 w[15];
    load_tw_inv<4, LOGN, 1, 0>(w, 0u, (int)((b << 4) + (uint32_t)i), tw);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 v = __ldcs(src + q);
        x[4 * q] = v.x;
        x[4 * q + 1] = v.y;
        x[4 * q + 2] = v.z;
        x[4 * q + 3] = v.w;
    }
    inv_stages_w<4, LOGN, 1, 0, F>(x, w, lc);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(&sm[ad.wv(q)]) = make_uint4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    __syncwarp();
    load_tw_inv<4, LOGN, 1, 4>(w, 0u, (int)b, tw);
    unroll16<0>([&](auto K) {
        constexpr int k = decltype(K)::value;
        x[k] = sm[ad.ws<k>()];
    });
    inv_stages_w<4, LOGN, 1, 4, F>(x, w, lc);
    uint32_t* dst = a.out + (size_t)row * N + (b << 8) + i;
#pragma unroll
    for (int k = 0; k < 16; ++k) dst[16 * k] = x[k];
}

// Inverse stages 8..15 of 16 columns of one row (N^-1 folded into stage 15), in place in out;
// canonical outputs.
template <int F>
__global__ void __launch_bounds__(THREADS, HEFX_2P_MINB) inv_cols_kernel(const Args2 a) {
    __shared__ uint32_t sm[16 * 256];
    griddep_wait();
    const uint32_t row = blockIdx.x / TASKS_PER_ROW;
    const uint32_t c0 = (blockIdx.x % TASKS_PER_ROW) * 16;
    const uint32_t limb = row % a.L;
    const LimbConst& lc = a.lc[limb];
    const uint2* tw = a.tw + (size_t)limb * N;
    const int c = threadIdx.x & 15, t = threadIdx.x >> 4;
    const ColAddr ad(c, t);
    uint32_t* base = a.out + (size_t)row * N + c0 + c;
    uint32_t x[16];
    uint2 w[15];
    load_tw_inv<4, LOGN, 1, 8>(w, 0u, t, tw);
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = __ldcg(base + 4096 * t + 256 * k);
    inv_stages_w<4, LOGN, 1, 8, F>(x, w, lc);
    unroll16<0>([&](auto K) {
        constexpr int k = decltype(K)::value;
        sm[ad.wb<k>()] = x[k];
    });
    __syncthreads();
    load_tw_inv<4, LOGN, 1, 12>(w, 0u, 0, tw);
    unroll16<0>([&](auto K) {
        constexpr int k = decltype(K)::value;
        x[k] = sm[ad.wa<k>()];
    });
    inv_stages_w<4, LOGN, 1, 12, F>(x, w, lc);
#pragma unroll
    for (int k = 0; k < 16; ++k) base[256 * t + 4096 * k] = x[k];
}

template <typename K>
cudaError_t launch2(K kern, const Args2& a, size_t rows, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)(rows * TASKS_PER_ROW));
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    // the set-up may overlap the stream's preceding kernel; every memory access follows
    // griddep_wait()
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int F>
cudaError_t launch_f(NttMode mode, const Args2& fa, const Args2& ia, size_t rows, cudaStream_t s) {
    if (mode == MODE_FWD) {
        cudaError_t e = launch2(fwd_cols_kernel<F>, fa, rows, s);
        if (e != cudaSuccess) return e;
        Args2 b = fa;
        b.in = fa.out;
        return launch2(fwd_rows_kernel<F>, b, rows, s);
    }
    cudaError_t e = launch2(inv_rows_kernel<F>, ia, rows, s);
    if (e != cudaSuccess) return e;
    Args2 b = ia;
    b.in = ia.out;
    return launch2(inv_cols_kernel<F>, b, rows, s);
}

}  // namespace cc2

bool ntt_cc_2p_supported(const hefx_params* p, NttMode mode) {
    return p->log2n == 16 && p->d_tw2_fwd && p->d_tw2_inv && (mode == MODE_FWD || mode == MODE_INV);
}

cudaError_t launch_ntt_cc_2p(const hefx_params* p, NttMode mode, const uint32_t* in, uint32_t* out, size_t rows,
                             cudaStream_t stream) {
    if (!ntt_cc_2p_supported(p, mode)) return cudaErrorNotSupported;
    if (rows == 0) return cudaSuccess;
    if (rows > (1u << 26)) return cudaErrorNotSupported;  // grid size stays in 32 bits
    cc2::Args2 fa = {in, out, p->d_tw2_fwd, p->d_lc, p->nlimbs};
    cc2::Args2 ia = {in, out, p->d_tw2_inv, p->d_lc, p->nlimbs};
    const bool lazy = p->max_prime < (1u << 28);
    return lazy ? cc2::launch_f<2>(mode, fa, ia, rows, stream) : cc2::launch_f<0>(mode, fa, ia, rows, stream);
}

}  // namespace hefx
