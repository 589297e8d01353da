// CUDA-core basis conversion (App. B, BConv) fed by TMA: the plain conversion
//
//   out_{n,j} = sum_i [a_{n,i} qhat_i^-1]_{q_i} [qhat_i]_{p_j}  mod p_j
//
// with the arithmetic of bconv.cu (step 1 a Shoup product, step 2 64-bit multiply-accumulates
// over 8 target limbs at a time, one Barrett reduction per output) and the memory side taken
// off the compute threads.  A persistent CTA streams tiles of 256 coefficients x L source limbs
// (one 2D tensor copy of L KiB each) through a ring of shared-memory stages (two per CTA,
// three CTAs per SM): one thread keeps the next copy in flight while eight warps convert the
// current one, a coefficient per thread, reading the residues from shared memory.  bconv.cu's direct-load
// kernel waits for one DRAM round trip per group of source limbs in every thread; here the
// copies of later tiles overlap the arithmetic of earlier ones.
#include <algorithm>

#include "bconv_common.h"
#include "modarith.cuh"
#include "tc_common.cuh"

namespace hefx {

namespace {

constexpr int kTile = 256;                 // coefficients per tile: one box of 256 words x L rows
// Stages per CTA and CTAs per SM (registers sized for them): measured on 16 x 24 -> 8 limbs of
// 2^16, 2 stages at 3 CTAs per SM 53.9 us, 3 at 2 56.0 us, 4 at 2 (one CTA fits) 64.2 us.
#ifndef HEFX_BCT_STAGES
#define HEFX_BCT_STAGES 2
#endif
#ifndef HEFX_BCT_MINB
#define HEFX_BCT_MINB 3
#endif
constexpr int kStages = HEFX_BCT_STAGES;   // tiles in flight per CTA
constexpr int kCompWarps = kTile / 32;     // one coefficient per compute thread
constexpr int kThreads = (kCompWarps + 1) * 32;
constexpr int kJ = 8;                      // target limbs per accumulation pass
constexpr uint32_t kMaxL = 48;             // a stage of 48 rows is 48 KiB

// Targets j0 .. j0+7 of one coefficient: acc[jj] = sum_i b_i [qhat_i]_{p_j}, b_i read from the
// stage (raw: this thread's column, stride kTile words).  STEP1: the stage holds a_i and b_i is
// computed here (Shoup product), and KEEP writes it back for the later target chunks.  Full
// groups of 8 source limbs first (loads at constant offsets), then the rest.
template <bool STEP1, bool KEEP>
__device__ __forceinline__ void accumulate(uint64_t (&acc)[kJ], uint32_t* raw, const BConvConst& c, uint32_t L,
                                           uint32_t j0) {
#pragma unroll
    for (int jj = 0; jj < kJ; ++jj) acc[jj] = 0;
    auto limb = [&](uint32_t i, uint32_t a) {
        uint32_t bi = a;
        if constexpr (STEP1) {
            const uint4 qc = *reinterpret_cast<const uint4*>(c.qpack[i]);  // q_i, qhat_i^-1, companion
            bi = csub(mul_shoup_lazy(a, qc.y, qc.z, qc.x), qc.x);
            if constexpr (KEEP) raw[i * kTile] = bi;  // this thread's own column
        }
        const uint4* row = reinterpret_cast<const uint4*>(&c.qhat_p[i * kBConvMaxLimbs + j0]);
        const uint4 r0 = row[0], r1 = row[1];
        const uint32_t cst[kJ] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
        for (int jj = 0; jj < kJ; ++jj) acc[jj] += (uint64_t)bi * cst[jj];
    };
    uint32_t i = 0;
    for (; i + 8 <= L; i += 8) {
        uint32_t a[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) a[g] = raw[(i + g) * kTile];
#pragma unroll
        for (int g = 0; g < 8; ++g) limb(i + g, a[g]);
    }
    for (; i < L; ++i) limb(i, raw[i * kTile]);
}

// Barrett-reduced outputs of targets j0 .. min(j0 + 8, Lp) - 1.
__device__ __forceinline__ void store_chunk(const uint64_t (&acc)[kJ], uint32_t* dst, const BConvConst& c, uint32_t Lp,
                                            uint32_t j0, uint32_t log2n) {
#pragma unroll
    for (int jj = 0; jj < kJ; ++jj) {
        const uint32_t j = j0 + jj;
        if (j < Lp) dst[(size_t)j << log2n] = barrett64(acc[jj], c.p[j], c.p_mu[j]);
    }
}

// Warps 0-7 convert (thread t: coefficient t of the tile), warp 8 lane 0 issues the copies.
// MULTI: more than 8 targets (several accumulation passes over the stage).
// Stage s is full when its copy has landed (full[s], transaction count) and empty when all
// eight compute warps have finished with it (empty[s], one arrival per warp).  Every wait is
// bounded: on a timeout the flag is set and the thread leaves its loop.
template <bool MULTI>
__global__ void __launch_bounds__(kThreads, HEFX_BCT_MINB)
    bconv_cc_tma_kernel(const __grid_constant__ CUtensorMap in_map, const BConvConst* __restrict__ gc,
                        uint32_t* __restrict__ out, uint32_t log2n, uint32_t batch, uint32_t* err) {
    extern __shared__ __align__(128) uint8_t stage_raw[];
    __shared__ __align__(16) BConvConst c;
    __shared__ uint64_t full[kStages], empty[kStages];
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        // the vectors, then the L used rows of the step 2 matrix (written at plan creation)
        const uint32_t L = __ldg(&gc->L);
        const uint32_t words = (uint32_t)(offsetof(BConvConst, qhat_p) / 4) + L * kBConvMaxLimbs;
        const uint4* s4 = reinterpret_cast<const uint4*>(gc);
        uint4* d4 = reinterpret_cast<uint4*>(&c);
        for (uint32_t k = tid; k < words / 4; k += kThreads) d4[k] = __ldg(s4 + k);
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], kCompWarps);
        }
        tc::fence_mbar_init();
    }
    __syncthreads();
    griddep_wait();  // the input may come from the stream's preceding kernel
    const uint32_t L = c.L, Lp = c.Lp;
    const uint32_t n = 1u << log2n, tiles_per_poly = n / kTile, ntiles = tiles_per_poly * batch;
    const uint32_t words = L * kTile;  // one stage

    if (warp == kCompWarps) {  // ---- copies
        if (lane == 0) {
            uint32_t it = 0;
            bool issued[kStages];
            uint32_t par[kStages];
            for (int s = 0; s < kStages; ++s) issued[s] = false;
            for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
                const uint32_t s = it % kStages, ph = (it / kStages) & 1u;
                if (!tc::mbar_wait(&empty[s], ph ^ 1u, err, tc::ERR_TIMEOUT_EMPTY)) break;
                const uint32_t b = t / tiles_per_poly, x0 = (t % tiles_per_poly) * kTile;
                tc::mbar_arrive_expect_tx(&full[s], words * 4u);
                tc::tma_load_2d(stage_raw + (size_t)s * words * 4u, &in_map, (int32_t)x0, (int32_t)(b * L), &full[s]);
                issued[s] = true;
                par[s] = ph;
            }
            // no copy may still be writing shared memory when the CTA exits
            for (int s = 0; s < kStages; ++s)
                if (issued[s]) tc::mbar_wait(&full[s], par[s], err, tc::ERR_TIMEOUT_FULL);
        }
        return;
    }
    // ---- conversion: thread tid takes coefficient tid of each tile
    uint32_t it = 0;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const uint32_t s = it % kStages, ph = (it / kStages) & 1u;
        if (!tc::mbar_wait(&full[s], ph, err, tc::ERR_TIMEOUT_FULL)) break;
        uint32_t* raw = reinterpret_cast<uint32_t*>(stage_raw) + (size_t)s * words + tid;
        const uint32_t b = t / tiles_per_poly, x = (t % tiles_per_poly) * kTile + tid;
        uint32_t* dst = out + ((size_t)b * Lp << log2n) + x;
        // the first 8 targets, with step 1 (kept in place when more targets follow)
        uint64_t acc[kJ];
        accumulate<true, MULTI>(acc, raw, c, L, 0);
        store_chunk(acc, dst, c, Lp, 0, log2n);
        if constexpr (MULTI) {
            for (uint32_t j0 = kJ; j0 < Lp; j0 += kJ) {
                accumulate<false, false>(acc, raw, c, L, j0);
                store_chunk(acc, dst, c, Lp, j0, log2n);
            }
            tc::fence_proxy_async_smem();  // the in-place writes before the stage's next copy
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&empty[s]);
    }
}

}  // namespace

cudaError_t launch_bconv_cc_tma(const hefx_bconv_plan* plan, const uint32_t* in, uint32_t* out, size_t batch,
                                uint32_t* err, cudaStream_t stream) {
    if (plan->log2n < 8 || plan->L > kMaxL || !err) return cudaErrorNotSupported;
    const uint32_t n = 1u << plan->log2n, L = plan->L;
    const size_t ntiles = (size_t)(n / kTile) * batch;
    if (ntiles == 0) return cudaSuccess;
    if (ntiles > 0xffffffffull || (size_t)batch * L > 0x7fffffffull) return cudaErrorInvalidValue;
    // the batch's source residues as a 2D array: rows (b, i) of n coefficients
    CUtensorMap in_map;
    if (!encode_map_2d(&in_map, CU_TENSOR_MAP_DATA_TYPE_UINT32, const_cast<uint32_t*>(in), n, batch * L,
                       (uint64_t)n * 4, kTile, L, CU_TENSOR_MAP_SWIZZLE_NONE))
        return cudaErrorNotSupported;  // no tensor-map encoder: the direct-load kernel runs
    const size_t smem = (size_t)kStages * L * kTile * 4;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    // per device and source count: the resident CTAs of the persistent grid
    static int resident[64][kMaxL + 1];
    static bool attr_set[64];
    if (dev < 0 || dev >= 64) dev = 0;
    if (!attr_set[dev]) {
        const int most = (int)((size_t)kStages * kMaxL * kTile * 4);
        e = cudaFuncSetAttribute(bconv_cc_tma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bconv_cc_tma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    if (resident[dev][L] == 0) {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bconv_cc_tma_kernel<true>, kThreads, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        resident[dev][L] = std::max(1, per_sm) * std::max(1, sms);
    }
    const unsigned grid = (unsigned)std::min<size_t>(ntiles, (size_t)resident[dev][L]);
    const BConvConst* gc = static_cast<const BConvConst*>(plan->d_const);
    if (plan->Lp > (uint32_t)kJ)
        return launch_pdl(bconv_cc_tma_kernel<true>, dim3(grid), dim3(kThreads), smem, stream, in_map, gc, out,
                          plan->log2n, (uint32_t)batch, err);
    return launch_pdl(bconv_cc_tma_kernel<false>, dim3(grid), dim3(kThreads), smem, stream, in_map, gc, out,
                      plan->log2n, (uint32_t)batch, err);
}

}  // namespace hefx
