// Tensor-core NTT, pipelined form: each matrix step of the layout-invariant 3-step NTT
// (Sec. IV-B) is one streamed digit GEMM
//
//     D[n][(out, o)] = sum_k Dig[n][k] * Cst[(out, o)][k],   k = (reduction index v, digit i)
//
// with the data digits as the A operand (128 data rows per CTA) and the BAT-compiled constant
// (Alg. 2, OfflineCompileLeft) as the B operand: 64 outputs x 4 chunks = 256 columns per tile.
// Data digits and constant chunks are both W bits (fp16-exact): W = 7 for moduli below 2^28,
// where partial sums stay below 4 * 256 * 127 * 127 < 2^24 for reduction lengths up to 256;
// W = 8 for moduli below 2^30, below 4 * 64 * 255 * 255 < 2^24 for reduction lengths up to 64
// (three-factor splits only).  The fp32 accumulation is exact; cvt.rni recovers the sums.
//
// GB300 mapping
//  - A (data digits, K-major) and B (constant, K-major) both arrive by TMA with the 128-byte
//    swizzle, 4 stages of 16 KiB + 32 KiB.  Each CTA loads its own constant stages: the
//    constant matrices of a limb (2 MiB per step at N = 2^16) stay resident in L2 while the
//    limb's data blocks stream past them.
//  - Two 256-column TMEM accumulators: the epilogue of one 64-output tile overlaps the MMAs
//    of the next.  The epilogue merges the 4 chunk sums (sum_o p_o 2^(W o) < 2^48), reduces
//    with one Montgomery REDC (2^32 folded into the constants), applies the twiddle or
//    Hadamard product and writes either the final residues or -- after a first step -- the
//    W-bit digits of the next step's A operand, already transposed where that step needs it.
//  - Persistent CTAs (as many as fit at once) walk the work items (limb, data block); the
//    two accumulators carry across items, so an item's last epilogue overlaps the next
//    item's MMAs.
//  - Warp roles: warp 0 TMA producer, warp 1 MMA issuer and TMEM owner, warps 2-17 epilogue
//    (four per TMEM lane quadrant, splitting the columns).  Every mbarrier wait is bounded.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "hefx_internal.h"
#include "host_nt.h"
#include "modarith.cuh"
#include "tc_common.cuh"

#ifndef HEFX_TC2_PDL
#define HEFX_TC2_PDL 1  // programmatic dependent launch of the digit GEMMs
#endif

namespace hefx {
namespace tc2 {

constexpr int BM = 128;                // data rows per CTA (MMA M)
constexpr int OUTS = 64;               // outputs per tile (the default tile; 32 is the other choice)
constexpr int KO = 4;                  // W-bit constant chunks
constexpr int BN = OUTS * KO;          // 256 (MMA N)
constexpr int BK = 64;                 // K elements per stage (128 bytes of fp16)
constexpr int STAGES = 4;
constexpr uint32_t A_BYTES = BM * BK * 2;  // 16 KiB
constexpr uint32_t B_BYTES = BN * BK * 2;  // 32 KiB
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
// warp 0 TMA, warp 1 MMA, warps 2-17 epilogue: four per TMEM lane quadrant, each on a quarter
// of the accumulator's columns (measured against two per quadrant: config 2 with 64 x 32 x 32,
// 147 / 147 us instead of 176 / 169 us per transform; the epilogue's dependent chain of TMEM
// read, conversions, REDC, twiddle load and digit stores needs the extra warps to hide latency)
constexpr int EPI_WARPS = 16;
constexpr int EPI_PARTS = EPI_WARPS / 4;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;
constexpr size_t SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + 256;

// Tile of TO outputs (TO * 4 accumulator columns; two accumulators in TMEM).
template <int TO>
struct Tile {
    static constexpr int BN = TO * KO;
    static constexpr uint32_t B_BYTES = BN * BK * 2;
    static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr uint32_t TMEM_COLS = 2 * BN < 32 ? 32 : 2 * BN;
    static constexpr size_t SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + 256;
};

// epilogue output: the next step's digits, or final residues [data row][output] or [output][data row]
enum : int { OUT_DIGITS = 0, OUT_U32_ROW_DATA = 1, OUT_U32_ROW_OUT = 2 };
// epilogue multiplier
enum : int { MUL_NONE = 0, MUL_TW = 1, MUL_HAD = 3, MUL_SQUARE = 4 };

struct Limb {
    uint32_t q, qinv_neg, r2, pad;
};

// One GEMM step of a matrix NTT: data row d (of DN per polynomial limb) times the constant gives
// OUT outputs o.  Index maps of the epilogue, with d split as (d mod D, d div D):
//  - twiddle (MUL_TW): tw[limb * twL + o twA + (d mod Dt) twB + (d div Dt) twC]
//  - next step's digits (OUT_DIGITS): row o rA + (d mod Dd) rB + (d div Dd) rC of orows rows per
//    polynomial limb, digit position 4 ((d mod Dd) kB + (d div Dd) kC) of 4 klen
//  - residues: out[d OUT + o] (OUT_U32_ROW_DATA) or out[o DN + d] (OUT_U32_ROW_OUT).
struct Args {
    uint32_t* out;          // u32 results [poly][limb][DN * OUT]
    uint16_t* out_digits;   // digits of the next step [poly][limb][orows][4 klen] (fp16 bits)
    const uint32_t* had;    // Hadamard operand, same layout as out
    const uint2* tw;        // Shoup twiddles, twL per limb
    const Limb* limbs;
    uint32_t* err;
    uint32_t L, batch;
    uint32_t DN;            // data rows per polynomial limb (A operand rows)
    uint32_t OUT;           // outputs per data row
    uint32_t K;             // 4 * reduction length
    uint32_t logDt, twA, twB, twC, twL;
    uint32_t logDd, rA, rB, rC, kB, kC, klen, orows;
};

template <int OUTK, int MUL, int TO, int W>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap, Args a) {
    constexpr int BN = Tile<TO>::BN, OUTS = TO;
    constexpr uint32_t STAGE_BYTES = Tile<TO>::STAGE_BYTES, TMEM_COLS = Tile<TO>::TMEM_COLS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;   // [2]
    uint64_t* acc_empty = acc_full + 2;    // [2]
    uint64_t* mma_done = acc_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);

    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // work items: (limb, data block of that limb).  A data block is 128 A rows of one limb: a
    // 128-row part of one polynomial's DN rows, or (DN < 128) the DN rows of PB = 128 / DN
    // consecutive polynomials; the digit buffers are limb-major ([limb][poly][DN][K]) so that
    // those rows are contiguous and share the limb's constant.  Consecutive items share the limb
    // (and so the L2-resident constant); CTAs walk the items with a stride.
    const uint32_t PB = a.DN >= BM ? 1u : BM / a.DN;
    const uint32_t blocks_per_poly = a.DN >= BM ? a.DN / BM : 1u;
    const uint32_t blocks_per_limb = a.DN >= BM ? a.batch * blocks_per_poly : (a.batch + PB - 1) / PB;
    const uint32_t items = a.L * blocks_per_limb;
    const uint32_t cid = blockIdx.x, nctas = gridDim.x;
    const uint32_t ntiles = a.OUT / OUTS, kstages = a.K / BK;
    auto item_rows = [&](uint32_t item, uint32_t& limb, uint32_t& poly0, uint32_t& drow0) {
        limb = item / blocks_per_limb;
        const uint32_t blk = item % blocks_per_limb;
        poly0 = a.DN >= BM ? blk / blocks_per_poly : blk * PB;
        drow0 = a.DN >= BM ? (blk % blocks_per_poly) * BM : 0u;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);  // the MMA commit that frees the stage
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_empty[b], 32 * EPI_WARPS);
        }
        tc::mbar_init(mma_done, 1);
        tc::fence_mbar_init();
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, TMEM_COLS);
    if (threadIdx.x == 32) {
        tc::prefetch_tmap(&amap);
        tc::prefetch_tmap(&bmap);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // Programmatic dependent launch: the set-up above touches only shared memory, TMEM and
    // the kernel's parameters; every global access below waits for the preceding kernel of the
    // stream to finish (a no-op when the launch did not allow the overlap).
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp == 0) {
        if (lane == 0) {  // ---- TMA producer
            uint32_t stage = 0, phase = 0;
            bool ok = true;
            for (uint32_t item = cid; item < items && ok; item += nctas) {
                uint32_t limb, poly0, drow0;
                item_rows(item, limb, poly0, drow0);
                const uint32_t a_row0 = (limb * a.batch + poly0) * a.DN + drow0;  // A rows: [limb][poly][DN]
                const uint32_t b_row0 = limb * a.OUT * KO;  // B rows: [limb][OUT x KO]
                for (uint32_t nt = 0; nt < ntiles && ok; ++nt)
                    for (uint32_t kc = 0; kc < kstages; ++kc) {
                        if (!tc::mbar_wait(&empty[stage], phase ^ 1u, a.err, tc::ERR_TIMEOUT_EMPTY)) {
                            ok = false;
                            break;
                        }
                        uint8_t* st = smem + stage * STAGE_BYTES;
                        tc::mbar_arrive_expect_tx(&full[stage], STAGE_BYTES);
                        tc::tma_load_2d(st, &amap, (int32_t)(kc * BK), (int32_t)a_row0, &full[stage]);
                        tc::tma_load_2d(st + A_BYTES, &bmap, (int32_t)(kc * BK), (int32_t)(b_row0 + nt * BN),
                                        &full[stage]);
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---- MMA issuer
            const uint32_t idesc = tc::idesc_f16_f32(BM, BN);
            uint32_t stage = 0, phase = 0, t = 0;  // t: tiles issued by this CTA so far
            bool ok = true;
            for (uint32_t item = cid; item < items && ok; item += nctas)
                for (uint32_t nt = 0; nt < ntiles && ok; ++nt, ++t) {
                    const uint32_t acc = t & 1;
                    if (t >= 2 && !tc::mbar_wait(&acc_empty[acc], ((t - 2) >> 1) & 1u, a.err, tc::ERR_TIMEOUT_ACC))
                        break;
                    tc::tc_fence_after();
                    for (uint32_t kc = 0; kc < kstages; ++kc) {
                        if (!tc::mbar_wait(&full[stage], phase, a.err, tc::ERR_TIMEOUT_FULL)) {
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                        const uint32_t ab = tc::smem_u32(smem + stage * STAGE_BYTES);
                        const uint32_t bb = ab + A_BYTES;
#pragma unroll
                        for (int ks = 0; ks < BK / 16; ++ks)
                            tc::mma_f16(tmem + acc * BN, tc::sw128_desc(ab + ks * 32), tc::sw128_desc(bb + ks * 32),
                                        idesc, (kc | ks) != 0);
                        tc::mma_commit(&empty[stage]);
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (ok) tc::mma_commit(&acc_full[acc]);
                }
            tc::mma_commit(mma_done);
            tc::mbar_wait(mma_done, 0, a.err, tc::ERR_TIMEOUT_ACC);
        }
    } else {  // ---- epilogue: warp % 4 is the TMEM lane quadrant, (warp - 2) / 4 the column slice
        const uint32_t quad = warp & 3, part = (warp - 2) >> 2;
        constexpr int SLICE = BN / EPI_PARTS;  // accumulator columns per epilogue warp
        static_assert(SLICE % 16 == 0, "whole 16-column TMEM reads per warp");
        uint32_t t = 0;
        for (uint32_t item = cid; item < items; item += nctas) {
            uint32_t limb, poly0, drow0;
            item_rows(item, limb, poly0, drow0);
            const uint32_t r = quad * 32 + lane;  // A row of the block held by this thread
            const uint32_t poly = poly0 + (PB > 1 ? r / a.DN : 0u);
            const uint32_t drow = PB > 1 ? r % a.DN : drow0 + r;  // data row within its polynomial limb
            const bool live = poly < a.batch;  // a block of several polynomials may run past the batch
            const uint32_t pl = (live ? poly : poly0) * a.L + limb;      // [poly][limb]: residues
            const uint32_t lp = limb * a.batch + (live ? poly : poly0);  // [limb][poly]: digits
            const Limb lc = a.limbs[limb];
            const size_t mat = (size_t)pl * a.DN * a.OUT;   // start of this polynomial limb
            // the data row's parts of the twiddle and digit index maps
            const uint32_t dt_lo = drow & ((1u << a.logDt) - 1u), dt_hi = drow >> a.logDt;
            const uint32_t dd_lo = drow & ((1u << a.logDd) - 1u), dd_hi = drow >> a.logDd;
            const uint2* twb = nullptr;
            if constexpr (MUL == MUL_TW)
                twb = a.tw + (size_t)limb * a.twL + (size_t)dt_lo * a.twB + (size_t)dt_hi * a.twC;
            uint16_t* dgb = nullptr;
            if constexpr (OUTK == OUT_DIGITS)
                dgb = a.out_digits +
                      ((size_t)lp * a.orows + (size_t)dd_lo * a.rB + (size_t)dd_hi * a.rC) * (4ull * a.klen) +
                      4ull * ((size_t)dd_lo * a.kB + (size_t)dd_hi * a.kC);
            bool ok = true;
            for (uint32_t nt = 0; nt < ntiles; ++nt, ++t) {
                const uint32_t acc = t & 1;
                if (!tc::mbar_wait(&acc_full[acc], (t >> 1) & 1u, a.err, tc::ERR_TIMEOUT_ACC)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
#pragma unroll 1
                for (int cb = (int)part * SLICE; cb < (int)(part + 1) * SLICE; cb += 16) {
                    uint32_t r[16];
                    tc::tmem_ld16(tmem + ((quad * 32) << 16) + acc * BN + cb, r);
                    tc::tmem_ld_wait();
                    const uint32_t out0 = nt * OUTS + cb / 4;
                    uint2 tw[4];
                    if constexpr (MUL == MUL_TW) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) tw[u] = __ldg(twb + (size_t)(out0 + u) * a.twA);
                    }
                    uint32_t res[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t p0 = __float2uint_rn(__uint_as_float(r[4 * u]));
                        const uint32_t p1 = __float2uint_rn(__uint_as_float(r[4 * u + 1]));
                        const uint32_t p2 = __float2uint_rn(__uint_as_float(r[4 * u + 2]));
                        const uint32_t p3 = __float2uint_rn(__uint_as_float(r[4 * u + 3]));
                        const uint64_t z = (uint64_t)p0 + ((uint64_t)p1 << W) + ((uint64_t)p2 << (2 * W)) +
                                           ((uint64_t)p3 << (3 * W));
                        const uint32_t zl = (uint32_t)z, zh = (uint32_t)(z >> 32);
                        uint32_t v = zh + __umulhi(zl * lc.qinv_neg, lc.q) + (zl != 0u);  // z 2^-32 mod q, [0, 2q)
                        const uint32_t out = out0 + u;
                        if constexpr (MUL == MUL_TW) {
                            v = mul_shoup_lazy(v, tw[u].x, tw[u].y, lc.q);
                        } else if constexpr (MUL == MUL_HAD) {
                            const uint32_t h = __ldg(a.had + mat + (size_t)drow * a.OUT + out);
                            v = mul_mont_lazy(mul_mont_lazy(v, h, lc.q, lc.qinv_neg), lc.r2, lc.q, lc.qinv_neg);
                        } else if constexpr (MUL == MUL_SQUARE) {
                            const uint32_t vc = csub(v, lc.q);
                            v = mul_mont_lazy(mul_mont_lazy(vc, vc, lc.q, lc.qinv_neg), lc.r2, lc.q, lc.qinv_neg);
                        }
                        res[u] = csub(v, lc.q);
                    }
                    if (!live) {
                    } else if constexpr (OUTK == OUT_DIGITS) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const uint2 d = tc::split_digits4<W>(res[u]);
                            *reinterpret_cast<uint2*>(dgb + (size_t)(out0 + u) * a.rA * (4ull * a.klen)) = d;
                        }
                    } else if constexpr (OUTK == OUT_U32_ROW_DATA) {
                        *reinterpret_cast<uint4*>(a.out + mat + (size_t)drow * a.OUT + out0) =
                            make_uint4(res[0], res[1], res[2], res[3]);
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u) a.out[mat + (size_t)(out0 + u) * a.DN + drow] = res[u];
                    }
                }
                tc::tc_fence_before();
                tc::mbar_arrive(&acc_empty[acc]);
            }
            if (!ok) break;
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// Matrix m = poly L + limb of the [poly][limb] data goes to digit matrix limb batch + poly (the
// digit buffers are limb-major, see gemm_kernel).
__device__ __forceinline__ size_t limb_major(size_t m, uint32_t L, uint32_t batch) {
    return (m % L) * batch + m / L;
}

// Digits of the first step's A operand where its rows are the data's rows (inverse step 1):
// 4 elements per thread, coalesced 16-byte loads and 32-byte stores.
template <int W>
__global__ void __launch_bounds__(256) digitize_kernel(const uint32_t* __restrict__ in, uint16_t* __restrict__ dig,
                                                       uint32_t R, uint32_t C, uint32_t L, uint32_t batch) {
    const size_t per = (size_t)R * C / 4;  // 4 elements per thread
    const size_t mats = (size_t)L * batch;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < mats * per; t += (size_t)gridDim.x * blockDim.x) {
        const size_t m = t / per, w = t % per;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(in + m * R * C) + w);
        const uint32_t r = (uint32_t)((w * 4) / C), c0 = (uint32_t)((w * 4) % C);
        const uint2 d0 = tc::split_digits4<W>(v.x), d1 = tc::split_digits4<W>(v.y);
        const uint2 d2 = tc::split_digits4<W>(v.z), d3 = tc::split_digits4<W>(v.w);
        uint4* o = reinterpret_cast<uint4*>(dig + limb_major(m, L, batch) * R * C * 4 + (size_t)r * (4 * C) + 4 * c0);
        o[0] = make_uint4(d0.x, d0.y, d1.x, d1.y);
        o[1] = make_uint4(d2.x, d2.y, d3.x, d3.y);
    }
}

// Digits of forward step 1's A operand, whose rows are the data's columns (K over its rows),
// on 64 x 64 tiles of the data matrix (R, C multiples of 64): each thread moves
// four 16-byte row pieces (16 KiB of loads per block), and the next tile's loads are issued
// before this tile's stores (persistent blocks).  Column c of the tile is 64 consecutive
// A-operand positions: one warp writes it as one 512-byte store, each lane the digits of two
// adjacent rows.  The odd row stride (65 words) limits the column reads to two-way conflicts.
__device__ __forceinline__ void load_tile64(const uint32_t* __restrict__ in, uint32_t R, uint32_t C, size_t tiles_per,
                                            size_t t, uint4 (&v)[4]) {
    const size_t m = t / tiles_per, w = t % tiles_per;
    const uint32_t r0 = (uint32_t)(w / (C / 64)) * 64, c0 = (uint32_t)(w % (C / 64)) * 64;
    const uint32_t* src = in + m * R * C;
#pragma unroll
    for (int k = 0; k < 4; ++k) {  // piece p = threadIdx + 256 k: row p / 16, columns 4 (p % 16) ..
        const uint32_t pc = threadIdx.x + 256u * k, r = pc >> 4, c = (pc & 15u) * 4;
        v[k] = __ldg(reinterpret_cast<const uint4*>(src + (size_t)(r0 + r) * C + c0 + c));
    }
}

// Column c of the data matrix becomes A row (c mod pr3) pr2 + c div pr3 (pr3 = 1: row c): the
// three-factor split orders its first step's rows (j2, j3) as (j3, j2) so that the step's
// epilogue writes its digits lane-contiguously.
template <int W>
__global__ void __launch_bounds__(256) digitize_t64_kernel(const uint32_t* __restrict__ in, uint16_t* __restrict__ dig,
                                                           uint32_t R, uint32_t C, uint32_t L, uint32_t batch,
                                                           uint32_t pr2, uint32_t pr3) {
    __shared__ uint32_t tile[64][65];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t mats = (size_t)L * batch;
    const size_t tiles_per = (size_t)(R / 64) * (C / 64), total = mats * tiles_per;
    size_t t = blockIdx.x;
    uint4 v[4];
    if (t < total) load_tile64(in, R, C, tiles_per, t, v);
    for (; t < total; t += gridDim.x) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t pc = threadIdx.x + 256u * k, r = pc >> 4, c = (pc & 15u) * 4;
            tile[r][c] = v[k].x;
            tile[r][c + 1] = v[k].y;
            tile[r][c + 2] = v[k].z;
            tile[r][c + 3] = v[k].w;
        }
        __syncthreads();
        if (t + gridDim.x < total) load_tile64(in, R, C, tiles_per, t + gridDim.x, v);  // in flight during the stores
        const size_t m = t / tiles_per, w = t % tiles_per;
        const uint32_t r0 = (uint32_t)(w / (C / 64)) * 64, c0 = (uint32_t)(w % (C / 64)) * 64;
        uint16_t* dst = dig + limb_major(m, L, batch) * R * C * 4;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t c = warp + 8 * k;  // this warp's column of the tile
            const uint2 lo = tc::split_digits4<W>(tile[2 * lane][c]), hi = tc::split_digits4<W>(tile[2 * lane + 1][c]);
            // A row of column c0 + c, K = 4 (r0 + 2 lane) .. + 7
            const uint32_t col = c0 + c, arow = (col % pr3) * pr2 + col / pr3;
            *reinterpret_cast<uint4*>(dst + (size_t)arow * (4 * R) + 4 * (r0 + 2 * lane)) =
                make_uint4(lo.x, lo.y, hi.x, hi.y);
        }
        __syncthreads();
    }
}

uint16_t half_bits_small(uint32_t d) {
    if (d == 0) return 0;
    int e = 31 - __builtin_clz(d);
    return (uint16_t)(((e + 15) << 10) | ((d << (10 - e)) & 0x3FFu));
}

}  // namespace tc2

// ------------------------------------------------------------------ host side

// Tables of one split of the matrix NTT (Sec. IV-B's layout-invariant form):
//  - two factors N = R x C: step 1 reduces over R (W1, twiddle T), step 2 over C (W3);
//  - three factors N = R1 x R2 x R3: step 1 as before with C = R2 R3, then the C-point cyclic
//    transform of each row (root w = psi^(2 R1)) as two steps: W2[p2][j2] = w^(R3 j2 brv(p2)),
//    twiddle T2[p2][j3] = w^(j3 brv(p2)), W3[p3][j3] = w^(R2 j3 brv(p3)); every output lands
//    at its bit-reversed position p1 R2 R3 + p2 R3 + p3 (the exponent j (2k + 1) mod 2N splits
//    over (j1, j2, j3) and (k1, k2, k3) with k = k1 + R1 k2 + R1 R2 k3).
// The inverse runs the mirror with the negated exponents and N^-1 folded into its last step.
struct Tc2Tables {
    uint32_t nsteps = 0;
    int W = 7;                        // digit and chunk width: 7 bits (moduli < 2^28) or 8 (< 2^30)
    uint32_t f[3] = {0, 0, 0};
    uint16_t* cst[6] = {};            // fp16 BAT digit matrices: forward steps, then inverse steps
    uint32_t cst_out[6] = {}, cst_v[6] = {};
    CUtensorMap bmaps[6][3];          // per matrix, per tile width 64 / 32 / 16 outputs
    uint2* twf[2] = {nullptr, nullptr};  // forward twiddles after steps 1 and 2
    uint2* twi[2] = {nullptr, nullptr};  // inverse twiddles after inverse steps 1 and 2
    tc2::Limb* limbs = nullptr;
    uint32_t* err = nullptr;
    uint16_t* dig1 = nullptr;
    uint16_t* dig3 = nullptr;
    size_t dig_elems = 0;
};

namespace {

int tile_index(uint32_t tile) { return tile >= 64 ? 0 : tile == 32 ? 1 : 2; }

}  // namespace

// The split a parameter set uses: log2 of its factors, from (tc_log2r, tc_log2r2).  Moduli of
// 29 or 30 bits take 8-bit digits, whose fp32 sums stay exact only for reduction lengths up to
// 64: their default is 64 x 64 at N = 2^12 and the three-factor split 64 x 32 x N/2048 (64 x 16
// x 16 at N = 2^14) from 2^14 on (N = 2^13 has no such split).
void tc2_split(const hefx_params* p, uint32_t f[3], uint32_t* nsteps) {
    const uint32_t logn = p->log2n;
    if (tc2_wide(p) && !p->tc_log2r2 && logn == 12) {
        f[0] = f[1] = 64;
        f[2] = 0;
        *nsteps = 2;
        return;
    }
    if (tc2_wide(p) && !p->tc_log2r2) {
        f[0] = 64;
        f[1] = logn >= 15 ? 32 : 16;
        f[2] = (1u << logn) / (64 * f[1]);
        *nsteps = 3;
        return;
    }
    const uint32_t l1 = p->tc_log2r ? p->tc_log2r : logn / 2;
    if (p->tc_log2r2) {
        f[0] = 1u << l1;
        f[1] = 1u << p->tc_log2r2;
        f[2] = 1u << (logn - l1 - p->tc_log2r2);
        *nsteps = 3;
    } else {
        f[0] = 1u << l1;
        f[1] = 1u << (logn - l1);
        f[2] = 0;
        *nsteps = 2;
    }
}

// Offline precompute: BAT digit matrices with W-bit input digits and W-bit output chunks,
// constants times 2^32 (Montgomery), rows (out, chunk) interleaved so that one output's four
// chunk sums land in four consecutive accumulator columns; Shoup twiddles.
cudaError_t tc2_prepare(hefx_params* p) {
    using namespace tc2;
    const uint32_t N = p->n, L = p->nlimbs;
    Tc2Tables* t = new Tc2Tables();
    tc2_split(p, t->f, &t->nsteps);
    t->W = tc2_wide(p) ? 8 : 7;
    const int W = t->W;
    const uint32_t ns = t->nsteps;
    const uint32_t R = t->f[0], C = N / R;  // step 1 and the rest (C = R2 R3 with three factors)
    const uint32_t R2 = t->f[1], R3 = ns == 3 ? t->f[2] : 1;
    // matrices: forward steps 0..ns-1, inverse steps ns..2ns-1 (outputs = reduction length)
    const uint32_t fw[3] = {R, ns == 3 ? R2 : C, R3};
    for (uint32_t k = 0; k < ns; ++k) {
        t->cst_out[k] = t->cst_v[k] = fw[k];
        t->cst_out[ns + k] = t->cst_v[ns + k] = fw[ns - 1 - k];  // inverse steps mirror the order
    }
    std::vector<std::vector<uint16_t>> hc(2 * ns);
    for (uint32_t m = 0; m < 2 * ns; ++m) hc[m].assign((size_t)L * t->cst_out[m] * KO * 4 * t->cst_v[m], 0);
    // twiddles per limb: forward T (N), then T2 (R2 R3); inverse T2inv (R2 R3), then Tinv (N)
    std::vector<uint2> hTf[2], hTi[2];
    hTf[0].resize((size_t)L * N);
    if (ns == 2) {
        hTi[0].resize((size_t)L * N);
    } else {
        hTf[1].resize((size_t)L * R2 * R3);
        hTi[0].resize((size_t)L * R2 * R3);
        hTi[1].resize((size_t)L * N);
    }
    std::vector<Limb> hl(L);
    auto work = [&](uint32_t l) {
        const uint64_t q = p->primes[l], psi = p->psi[l], twoN = 2ull * N;
        std::vector<uint64_t> pw(twoN);
        pw[0] = 1;
        for (uint64_t e = 1; e < twoN; ++e) pw[e] = mul_mod(pw[e - 1], psi, q);
        auto P = [&](uint64_t e) { return pw[e % twoN]; };
        auto Pn = [&](uint64_t e) { return pw[(twoN - e % twoN) % twoN]; };
        const uint64_t r32 = ((uint64_t)1 << 32) % q, ninv = inv_mod(N % q, q);
        hl[l] = {(uint32_t)q, neg_inv_pow2_32((uint32_t)q), (uint32_t)mul_mod(r32, r32, q), 0};
        auto put = [&](uint32_t m, uint32_t out, uint32_t v, uint64_t w) {
            const uint32_t K = 4 * t->cst_v[m];
            uint64_t c = mul_mod(w, r32, q);
            for (uint32_t i = 0; i < 4; ++i) {
                for (int o = 0; o < KO; ++o) {
                    const uint32_t chunk = (uint32_t)((c >> (W * o)) & ((1u << W) - 1u));
                    hc[m][(((size_t)l * t->cst_out[m] + out) * KO + o) * K + v * 4 + i] = half_bits_small(chunk);
                }
                c = (c << W) % q;
            }
        };
        auto shoup2 = [&](uint64_t w) { return make_uint2((uint32_t)w, shoup(w, q)); };
        const int logR = 31 - __builtin_clz(R);
        // step 1 over R (both forms): W1[p1][j1] = psi^(C j1 (2 brv(p1) + 1)); its inverse
        // (the last inverse step) with N^-1; twiddle T[p1][j] = psi^(j (2 brv(p1) + 1)), the
        // inverse one stored transposed [j][p1]
        for (uint32_t p1 = 0; p1 < R; ++p1) {
            const uint64_t kodd = 2ull * bit_reverse(p1, logR) + 1;
            for (uint32_t j1 = 0; j1 < R; ++j1) {
                put(0, p1, j1, P((uint64_t)C * j1 * kodd));
                put(2 * ns - 1, j1, p1, mul_mod(ninv, Pn((uint64_t)C * j1 * kodd), q));
            }
            for (uint32_t j = 0; j < C; ++j) {
                // three factors: the first step's data rows come in the order (j3, j2)
                const uint32_t jr = ns == 3 ? (j % R3) * R2 + j / R3 : j;
                hTf[0][(size_t)l * N + (size_t)p1 * C + jr] = shoup2(P((uint64_t)j * kodd));
                hTi[ns - 2][(size_t)l * N + (size_t)j * R + p1] = shoup2(Pn((uint64_t)j * kodd));
            }
        }
        if (ns == 2) {
            // C-point cyclic step: W3[p2][j2] = psi^(2R j2 brv(p2)); inverse first step mirror
            const int logC = 31 - __builtin_clz(C);
            for (uint32_t p2 = 0; p2 < C; ++p2) {
                const uint64_t kb = bit_reverse(p2, logC);
                for (uint32_t j2 = 0; j2 < C; ++j2) {
                    put(1, p2, j2, P(2ull * R * j2 * kb));
                    put(2, j2, p2, Pn(2ull * R * j2 * kb));
                }
            }
        } else {
            // the C-point cyclic transform (w = psi^(2R)) as R2 x R3
            const int log2 = 31 - __builtin_clz(R2), log3 = 31 - __builtin_clz(R3);
            for (uint32_t p2 = 0; p2 < R2; ++p2) {
                const uint64_t b2 = bit_reverse(p2, log2);
                for (uint32_t j2 = 0; j2 < R2; ++j2) {
                    put(1, p2, j2, P(2ull * R * R3 * j2 * b2));   // W2
                    put(4, j2, p2, Pn(2ull * R * R3 * j2 * b2));  // inverse step 2: V2[j2][p2]
                }
                for (uint32_t j3 = 0; j3 < R3; ++j3) {
                    hTf[1][(size_t)l * R2 * R3 + (size_t)p2 * R3 + j3] = shoup2(P(2ull * R * j3 * b2));
                    hTi[0][(size_t)l * R2 * R3 + (size_t)j3 * R2 + p2] = shoup2(Pn(2ull * R * j3 * b2));
                }
            }
            for (uint32_t p3 = 0; p3 < R3; ++p3) {
                const uint64_t b3 = bit_reverse(p3, log3);
                for (uint32_t j3 = 0; j3 < R3; ++j3) {
                    put(2, p3, j3, P(2ull * R * R2 * j3 * b3));   // W3
                    put(3, j3, p3, Pn(2ull * R * R2 * j3 * b3));  // inverse step 1: V3[j3][p3]
                }
            }
        }
    };
    {
        std::vector<std::thread> th;
        const uint32_t nth = std::max(1u, std::min(L, std::thread::hardware_concurrency()));
        for (uint32_t w = 0; w < nth; ++w)
            th.emplace_back([&, w] {
                for (uint32_t l = w; l < L; l += nth) work(l);
            });
        for (auto& x : th) x.join();
    }
    cudaError_t e = cudaSuccess;
    for (uint32_t m = 0; m < 2 * ns && e == cudaSuccess; ++m) {
        e = cudaMalloc(&t->cst[m], hc[m].size() * 2);
        if (e == cudaSuccess) e = cudaMemcpy(t->cst[m], hc[m].data(), hc[m].size() * 2, cudaMemcpyHostToDevice);
        for (int w = 0; w < 3 && e == cudaSuccess; ++w) {
            const uint32_t tile = 64u >> w;
            if (tile > t->cst_out[m]) continue;
            if (!encode_map_2d(&t->bmaps[m][w], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, t->cst[m], 4ull * t->cst_v[m],
                               (uint64_t)L * t->cst_out[m] * KO, 8ull * t->cst_v[m], BK, tile * KO,
                               CU_TENSOR_MAP_SWIZZLE_128B))
                e = cudaErrorInvalidValue;
        }
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        if (hTf[k].empty()) continue;
        e = cudaMalloc(&t->twf[k], hTf[k].size() * sizeof(uint2));
        if (e == cudaSuccess)
            e = cudaMemcpy(t->twf[k], hTf[k].data(), hTf[k].size() * sizeof(uint2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&t->twi[k], hTi[k].size() * sizeof(uint2));
        if (e == cudaSuccess)
            e = cudaMemcpy(t->twi[k], hTi[k].data(), hTi[k].size() * sizeof(uint2), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&t->limbs, L * sizeof(Limb));
    if (e == cudaSuccess) e = cudaMemcpy(t->limbs, hl.data(), L * sizeof(Limb), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&t->err, 4);
    if (e == cudaSuccess) e = cudaMemset(t->err, 0, 4);
    p->tc2 = t;
    if (e != cudaSuccess) tc2_free(p);
    return e;
}

void tc2_free(hefx_params* p) {
    Tc2Tables* t = p->tc2;
    if (!t) return;
    for (int m = 0; m < 6; ++m)
        if (t->cst[m]) cudaFree(t->cst[m]);
    for (int k = 0; k < 2; ++k) {
        if (t->twf[k]) cudaFree(t->twf[k]);
        if (t->twi[k]) cudaFree(t->twi[k]);
    }
    if (t->limbs) cudaFree(t->limbs);
    if (t->err) cudaFree(t->err);
    if (t->dig1) cudaFree(t->dig1);
    if (t->dig3) cudaFree(t->dig3);
    delete t;
    p->tc2 = nullptr;
}

uint32_t* tc2_err(const hefx_params* p) { return p->tc2 ? p->tc2->err : nullptr; }

namespace {

cudaError_t ensure_workspace(Tc2Tables* t, size_t elems) {
    if (t->dig_elems >= elems) return cudaSuccess;
    cudaError_t e = cudaDeviceSynchronize();  // the old buffers may still be in use
    if (e != cudaSuccess) return e;
    if (t->dig1) cudaFree(t->dig1);
    if (t->dig3) cudaFree(t->dig3);
    t->dig1 = t->dig3 = nullptr;
    t->dig_elems = 0;
    e = cudaMalloc(&t->dig1, elems * 8);
    if (e == cudaSuccess) e = cudaMalloc(&t->dig3, elems * 8);
    if (e == cudaSuccess) t->dig_elems = elems;
    return e;
}

template <int OUTK, int MUL, int TO, int W>
cudaError_t launch_gemm_t(const CUtensorMap& amap, const CUtensorMap& bmap, const tc2::Args& g, cudaStream_t s) {
    using namespace tc2;
    auto kern = gemm_kernel<OUTK, MUL, TO, W>;
    constexpr size_t SMEM_BYTES = Tile<TO>::SMEM_BYTES;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    const uint32_t pb = g.DN >= BM ? 1u : BM / g.DN;  // as in the kernel
    const uint32_t items = g.L * (g.DN >= BM ? g.batch * (g.DN / BM) : (g.batch + pb - 1) / pb);
    // persistent: as many CTAs as can be resident at once (one per SM: the pipeline's shared
    // memory), cached per device
    static int max_ctas[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!max_ctas[dev & 63]) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, SMEM_BYTES) != cudaSuccess ||
            per_sm <= 0)
            per_sm = 1;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
        max_ctas[dev & 63] = per_sm * sms;
    }
    cfg.gridDim = dim3(std::min<uint32_t>(items, (uint32_t)max_ctas[dev & 63]));
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = s;
    // the set-up of this GEMM may overlap the tail of the stream's preceding kernel
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = HEFX_TC2_PDL;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, amap, bmap, g);
}

template <int OUTK, int MUL, int W>
cudaError_t launch_gemm_w(const CUtensorMap* bmaps, uint32_t tile, const CUtensorMap& amap, const tc2::Args& g,
                          cudaStream_t s) {
    if (tile >= 64) return launch_gemm_t<OUTK, MUL, 64, W>(amap, bmaps[0], g, s);
    if (tile == 32) return launch_gemm_t<OUTK, MUL, 32, W>(amap, bmaps[1], g, s);
    return launch_gemm_t<OUTK, MUL, 16, W>(amap, bmaps[2], g, s);
}

template <int OUTK, int MUL>
cudaError_t launch_gemm(const CUtensorMap* bmaps, uint32_t tile, int W, const CUtensorMap& amap, const tc2::Args& g,
                        cudaStream_t s) {
    return W == 8 ? launch_gemm_w<OUTK, MUL, 8>(bmaps, tile, amap, g, s)
                  : launch_gemm_w<OUTK, MUL, 7>(bmaps, tile, amap, g, s);
}

int ilog2(uint32_t x) { return 31 - __builtin_clz(x); }

// One GEMM step: constant matrix m, A digits `adig` ([poly][limb][DN][4 V]); output per outk.
struct StepSpec {
    uint32_t m, DN;
    int outk, mul;
    const uint2* tw;
    uint32_t Dt, twA, twB, twC, twL;
    uint32_t Dd, rA, rB, rC, kB, kC, klen, orows;
};

cudaError_t run_step(const hefx_params* p, const StepSpec& st, const uint16_t* adig, uint16_t* odig, uint32_t* out,
                     const uint32_t* had, size_t batch, cudaStream_t s) {
    using namespace tc2;
    const Tc2Tables* t = p->tc2;
    Args g;
    memset(&g, 0, sizeof g);
    g.out = out;
    g.out_digits = odig;
    g.had = had;
    g.tw = st.tw;
    g.limbs = t->limbs;
    g.err = t->err;
    g.L = p->nlimbs;
    g.batch = (uint32_t)batch;
    g.DN = st.DN;
    g.OUT = t->cst_out[st.m];
    g.K = 4 * t->cst_v[st.m];
    g.logDt = ilog2(st.Dt ? st.Dt : 1);
    g.twA = st.twA;
    g.twB = st.twB;
    g.twC = st.twC;
    g.twL = st.twL;
    g.logDd = ilog2(st.Dd ? st.Dd : 1);
    g.rA = st.rA;
    g.rB = st.rB;
    g.rC = st.rC;
    g.kB = st.kB;
    g.kC = st.kC;
    g.klen = st.klen;
    g.orows = st.orows;
    CUtensorMap amap;
    if (!encode_map_2d(&amap, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, const_cast<uint16_t*>(adig), g.K,
                       (uint64_t)batch * g.L * g.DN, 2ull * g.K, BK, BM, CU_TENSOR_MAP_SWIZZLE_128B))
        return cudaErrorInvalidValue;
    const uint32_t tile = std::min<uint32_t>(p->tc_tile == 32 ? 32u : 64u, g.OUT);
    const CUtensorMap* b3 = t->bmaps[st.m];
    const int W = t->W;
    if (st.outk == OUT_DIGITS) return launch_gemm<OUT_DIGITS, MUL_TW>(b3, tile, W, amap, g, s);
    if (st.outk == OUT_U32_ROW_OUT) return launch_gemm<OUT_U32_ROW_OUT, MUL_NONE>(b3, tile, W, amap, g, s);
    switch (st.mul) {
        case MUL_HAD: return launch_gemm<OUT_U32_ROW_DATA, MUL_HAD>(b3, tile, W, amap, g, s);
        case MUL_SQUARE: return launch_gemm<OUT_U32_ROW_DATA, MUL_SQUARE>(b3, tile, W, amap, g, s);
        default: return launch_gemm<OUT_U32_ROW_DATA, MUL_NONE>(b3, tile, W, amap, g, s);
    }
}

cudaError_t digitize(const hefx_params* p, const uint32_t* in, uint16_t* dig, bool trans, uint32_t R, uint32_t C,
                     size_t batch, cudaStream_t s, uint32_t pr2 = 1, uint32_t pr3 = 1) {
    const size_t mats = batch * p->nlimbs;
    const size_t work = mats * p->n / 4;
    const unsigned grid = (unsigned)std::min<size_t>((work + 255) / 256, (size_t)1 << 20);
    if (trans) {  // R, C multiples of 64
        const size_t tiles = mats * (R / 64) * (C / 64);
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // persistent: 8 blocks of 256 threads per SM (16.6 KiB of shared memory each)
        const unsigned blocks = (unsigned)std::min<size_t>(tiles, (size_t)sms * 8);
        const uint32_t L = p->nlimbs, B = (uint32_t)batch;
        if (p->tc2->W == 8)
            tc2::digitize_t64_kernel<8><<<blocks, 256, 0, s>>>(in, dig, R, C, L, B, pr2, pr3);
        else
            tc2::digitize_t64_kernel<7><<<blocks, 256, 0, s>>>(in, dig, R, C, L, B, pr2, pr3);
    } else if (p->tc2->W == 8) {
        tc2::digitize_kernel<8><<<grid, 256, 0, s>>>(in, dig, R, C, p->nlimbs, (uint32_t)batch);
    } else {
        tc2::digitize_kernel<7><<<grid, 256, 0, s>>>(in, dig, R, C, p->nlimbs, (uint32_t)batch);
    }
    return cudaGetLastError();
}

}  // namespace

// forward: digits of the columns -> [step 1 over R, x T] -> digits -> ... -> residues in
// bit-reversed order (two or three steps; see Tc2Tables)
cudaError_t tc2_forward(hefx_params* p, const uint32_t* in, uint32_t* out, int mul, const uint32_t* had, size_t batch,
                        cudaStream_t s) {
    using namespace tc2;
    Tc2Tables* t = p->tc2;
    const uint32_t N = p->n, R = t->f[0], C = N / R;
    cudaError_t e = ensure_workspace(t, batch * p->nlimbs * (size_t)N);
    if (t->nsteps == 2) {
        if (e == cudaSuccess) e = digitize(p, in, t->dig1, true, R, C, batch, s);
        const StepSpec s1 = {0, C, OUT_DIGITS, MUL_TW, t->twf[0], C, C, 1, 0, N, C, 1, 0, 0, 1, 0, C, R};
        const StepSpec s2 = {1, R, OUT_U32_ROW_DATA, mul, nullptr, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0};
        if (e == cudaSuccess) e = run_step(p, s1, t->dig1, t->dig3, nullptr, nullptr, batch, s);
        if (e == cudaSuccess) e = run_step(p, s2, t->dig3, nullptr, out, had, batch, s);
        return e;
    }
    const uint32_t R2 = t->f[1], R3 = t->f[2];
    if (e == cudaSuccess) e = digitize(p, in, t->dig1, true, R, C, batch, s, R2, R3);
    // step 1: data row j3 R2 + j2 (column j = j2 R3 + j3, reordered by the digit split; T stored
    // in that order) -> digits of row (p1, j3), position j2 (lanes write consecutive positions)
    const StepSpec s1 = {0, C, OUT_DIGITS, MUL_TW, t->twf[0], C, C, 1, 0, N, R2, R3, 0, 1, 1, 0, R2, R * R3};
    // step 2: data row (p1, j3), output p2 -> digits of row (p1, p2), position j3
    const StepSpec s2 = {1, R * R3, OUT_DIGITS, MUL_TW, t->twf[1], R3, R3, 1, 0, R2 * R3, R3, 1, 0, R2, 1, 0, R3, R * R2};
    // step 3: data row (p1, p2), outputs p3 -> residue at p1 R2 R3 + p2 R3 + p3
    const StepSpec s3 = {2, R * R2, OUT_U32_ROW_DATA, mul, nullptr, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = run_step(p, s1, t->dig1, t->dig3, nullptr, nullptr, batch, s);
    if (e == cudaSuccess) e = run_step(p, s2, t->dig3, t->dig1, nullptr, nullptr, batch, s);
    if (e == cudaSuccess) e = run_step(p, s3, t->dig1, nullptr, out, had, batch, s);
    return e;
}

// inverse: digits of the rows -> the mirror steps (twiddles inverted, N^-1 in the last) ->
// residues in natural order
cudaError_t tc2_inverse(hefx_params* p, const uint32_t* in, uint32_t* out, size_t batch, cudaStream_t s) {
    using namespace tc2;
    Tc2Tables* t = p->tc2;
    const uint32_t N = p->n, R = t->f[0], C = N / R;
    cudaError_t e = ensure_workspace(t, batch * p->nlimbs * (size_t)N);
    if (t->nsteps == 2) {
        if (e == cudaSuccess) e = digitize(p, in, t->dig1, false, R, C, batch, s);
        // data row p1, output j2; twiddle stored [j2][p1]; digits of row j2, position p1
        const StepSpec s1 = {2, R, OUT_DIGITS, MUL_TW, t->twi[0], R, R, 1, 0, N, R, 1, 0, 0, 1, 0, R, C};
        const StepSpec s2 = {3, C, OUT_U32_ROW_OUT, MUL_NONE, nullptr, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0};
        if (e == cudaSuccess) e = run_step(p, s1, t->dig1, t->dig3, nullptr, nullptr, batch, s);
        if (e == cudaSuccess) e = run_step(p, s2, t->dig3, nullptr, out, nullptr, batch, s);
        return e;
    }
    const uint32_t R2 = t->f[1], R3 = t->f[2];
    if (e == cudaSuccess) e = digitize(p, in, t->dig1, false, R * R2, R3, batch, s);
    // inverse step 1: data row (p1, p2), output j3; twiddle T2inv stored [j3][p2]; digits of
    // row (j3, p1), position p2
    const StepSpec s1 = {3, R * R2, OUT_DIGITS, MUL_TW, t->twi[0], R2, R2, 1, 0, R2 * R3, R2, R, 0, 1, 1, 0, R2, R3 * R};
    // inverse step 2: data row (j3, p1), output j2; twiddle Tinv[j2 R3 + j3][p1]; digits of row
    // j = j2 R3 + j3, position p1 (lanes: consecutive p1 in both)
    const StepSpec s2 = {4, R3 * R, OUT_DIGITS, MUL_TW, t->twi[1], R3 * R, R3 * R, 1, 0, N, R, R3, 0, 1, 1, 0, R, C};
    // inverse step 3: data row j, output j1 (N^-1 folded) -> residue j1 C + j
    const StepSpec s3 = {5, C, OUT_U32_ROW_OUT, MUL_NONE, nullptr, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = run_step(p, s1, t->dig1, t->dig3, nullptr, nullptr, batch, s);
    if (e == cudaSuccess) e = run_step(p, s2, t->dig3, t->dig1, nullptr, nullptr, batch, s);
    if (e == cudaSuccess) e = run_step(p, s3, t->dig1, nullptr, out, nullptr, batch, s);
    return e;
}

// c = INTT(NTT(a) o NTT(b)); c may alias a and/or b
cudaError_t tc2_polymul(hefx_params* p, const uint32_t* a, const uint32_t* b, uint32_t* c, size_t batch,
                        cudaStream_t s) {
    using namespace tc2;
    cudaError_t e;
    if (a == b) {
        e = tc2_forward(p, a, c, MUL_SQUARE, nullptr, batch, s);
    } else {
        if (c == b) std::swap(a, b);
        e = tc2_forward(p, a, c, MUL_NONE, nullptr, batch, s);            // c = NTT(a)
        if (e == cudaSuccess) e = tc2_forward(p, b, c, MUL_HAD, c, batch, s);  // c = NTT(b) o c
    }
    if (e == cudaSuccess) e = tc2_inverse(p, c, c, batch, s);
    return e;
}

}  // namespace hefx
