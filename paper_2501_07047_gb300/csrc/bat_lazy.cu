// VecModMul with the BAT lazy modular reduction on the tensor cores (the paper's "BAT for
// Modular Reduction" appendix; evaluated, on the TPU, in the reduction ablation of Sec. V-F).
//
// For z = x y mod q the 64-bit product psum = sum_{j < 8} c_j 2^(8j) (bytes c_j) splits into
// its low 32 bits and the high bytes c_4..c_7, and
//
//     psum = low + sum_{j < 4} c_{4+j} 2^(8(4+j))
//          = low + sum_{k < 4} ( sum_{j < 4} c_{4+j} LC_{j,k} ) 2^(8k)   (mod q),
//
// with LC_j = 2^(8(4+j)) mod q and LC_{j,k} its bytes: a (elements x 4) x (4 x 4) byte matrix
// product.  Here it is one tcgen05.mma per 128 elements: the high bytes are the A operand (one
// row per element, fp16, K padded to 16), the byte matrix LC the B operand (N padded to 16),
// fp32 accumulation (each sum < 4 * 255 * 255 < 2^24, exact).  The merged value
// low + sum_k s_k 2^(8k) < 2^44 is congruent to psum and takes one final Barrett reduction to
// the canonical residue, so the results equal the CUDA-core reductions' bit for bit.
//
// GB300 mapping: a persistent CTA of 128 threads takes 512 elements per step (thread t owns
// elements 4t..4t+3 through 16-byte loads and stores): four 128-row A tiles (K-major, 128-byte
// swizzle, 16 KiB each) and one 16-row B tile in shared memory, four MMAs into 64 TMEM columns
// (sub-tile u in columns 16u..16u+3), then every thread reads its lane's four sums.  The next
// step's loads are issued before the MMAs are waited for.  The wait is bounded (error flag).
#include "hefx_internal.h"
#include "modarith.cuh"
#include "tc_common.cuh"

namespace hefx {
namespace bat {

constexpr int THREADS = 128;
constexpr int SUB = 4;                      // 128-row sub-tiles per step (elements per thread)
constexpr uint32_t TILE = THREADS * SUB;    // 512 elements per step
constexpr uint32_t A_BYTES = 128 * 128;     // 128 rows x 128 bytes (64 fp16 of K; 4 used)
constexpr uint32_t B_BYTES = 16 * 128;      // 16 rows (outputs k; 4 used) x 128 bytes
constexpr uint32_t TMEM_COLS = 64;          // 4 sub-tiles x 16 columns
constexpr size_t SMEM_BYTES = 1024 + SUB * A_BYTES + B_BYTES + 64;
constexpr uint32_t ERR_TIMEOUT_MMA = 4;     // error code: an MMA did not complete in time

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
}

// The four high bytes of psum as fp16 in the first 8 K-slots of an A row (the rest zero).
__device__ __forceinline__ uint4 high_bytes_row(uint64_t psum) {
    const uint32_t hi = (uint32_t)(psum >> 32);
    return make_uint4(tc::digits_to_half2(hi & 255u, (hi >> 8) & 255u),
                      tc::digits_to_half2((hi >> 16) & 255u, hi >> 24), 0u, 0u);
}

__device__ __forceinline__ uint32_t barrett64(uint64_t z, const LimbConst& c) {
    const uint64_t mu = ((uint64_t)c.bar_hi << 32) | c.bar_lo;  // floor(2^64 / q)
    return csub((uint32_t)(z - __umul64hi(z, mu) * c.q), c.q);   // z < 2^64: remainder < 2q
}

__global__ void __launch_bounds__(THREADS) vec_mod_mul_bat_kernel(const LimbConst* __restrict__ lc, uint32_t L,
                                                                  uint32_t log2n, size_t nsteps,
                                                                  const uint4* __restrict__ x,
                                                                  const uint4* __restrict__ y, uint4* __restrict__ z,
                                                                  uint32_t* err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* a_tiles = sm;
    uint8_t* b_tile = sm + SUB * A_BYTES;
    uint64_t* bar = reinterpret_cast<uint64_t*>(b_tile + B_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
    const uint32_t t = threadIdx.x, warp = t >> 5;

    // zero both operands once: only the first 16-byte chunk of each used row is rewritten
    for (uint32_t i = t; i < (SUB * A_BYTES + B_BYTES) / 16; i += THREADS)
        reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
    if (warp == 0) tc::tmem_alloc(tmem_slot, TMEM_COLS);
    if (t == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t taddr = *tmem_slot;
    const uint32_t idesc = tc::idesc_f16_f32(128, 16);
    const uint32_t a_addr = tc::smem_u32(a_tiles), b_addr = tc::smem_u32(b_tile);

    uint32_t phase = 0, cur_limb = 0xFFFFFFFFu;
    size_t step = blockIdx.x;
    uint4 xv = make_uint4(0, 0, 0, 0), yv = xv;
    if (step < nsteps) {
        xv = __ldg(x + step * THREADS + t);
        yv = __ldg(y + step * THREADS + t);
    }
    for (; step < nsteps; step += gridDim.x) {
        const uint32_t limb = (uint32_t)(((step * TILE) >> log2n) % L);  // N >= 512: one limb per step
        const LimbConst c = lc[limb];
        const uint32_t xs[SUB] = {xv.x, xv.y, xv.z, xv.w}, ys[SUB] = {yv.x, yv.y, yv.z, yv.w};
        uint32_t low[SUB];
#pragma unroll
        for (int u = 0; u < SUB; ++u) {
            const uint64_t psum = (uint64_t)xs[u] * ys[u];
            low[u] = (uint32_t)psum;
            *reinterpret_cast<uint4*>(a_tiles + u * A_BYTES + tc::sw128_offset(t, 0)) = high_bytes_row(psum);
        }
        if (limb != cur_limb) {  // B row k: byte k of LC_0..LC_3 (uniform across the CTA)
            if (t < 4) {
                uint64_t lcj = ((uint64_t)1 << 32) % c.q;  // LC_0 = 2^32 mod q
                uint32_t bytes[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    bytes[j] = (uint32_t)(lcj >> (8 * t)) & 255u;
                    lcj = (lcj << 8) % c.q;  // LC_{j+1} = 2^8 LC_j mod q
                }
                *reinterpret_cast<uint4*>(b_tile + tc::sw128_offset(t, 0)) =
                    make_uint4(tc::digits_to_half2(bytes[0], bytes[1]), tc::digits_to_half2(bytes[2], bytes[3]), 0u, 0u);
            }
            cur_limb = limb;
        }
        tc::fence_proxy_async_smem();  // the operand writes before the tensor cores read them
        __syncthreads();
        if (t == 0) {
            tc::tc_fence_after();
#pragma unroll
            for (int u = 0; u < SUB; ++u)
                tc::mma_f16(taddr + 16 * u, tc::sw128_desc(a_addr + u * A_BYTES), tc::sw128_desc(b_addr), idesc, 0);
            tc::mma_commit(bar);
        }
        // the next step's operands load while the MMAs run
        const size_t next = step + gridDim.x;
        if (next < nsteps) {
            xv = __ldg(x + next * THREADS + t);
            yv = __ldg(y + next * THREADS + t);
        }
        tc::mbar_wait(bar, phase, err, ERR_TIMEOUT_MMA);
        phase ^= 1u;
        tc::tc_fence_after();
        uint32_t s[SUB][4];
#pragma unroll
        for (int u = 0; u < SUB; ++u) tmem_ld4(taddr + ((warp * 32u) << 16) + 16 * u, s[u]);
        tc::tmem_ld_wait();
        uint32_t out[SUB];
#pragma unroll
        for (int u = 0; u < SUB; ++u) {
            const uint64_t merged = (uint64_t)low[u] + tc::acc_to_u32(s[u][0]) + ((uint64_t)tc::acc_to_u32(s[u][1]) << 8) +
                                    ((uint64_t)tc::acc_to_u32(s[u][2]) << 16) +
                                    ((uint64_t)tc::acc_to_u32(s[u][3]) << 24);
            out[u] = barrett64(merged, c);
        }
        z[step * THREADS + t] = make_uint4(out[0], out[1], out[2], out[3]);
        tc::tc_fence_before();
        __syncthreads();  // operands and accumulators are rewritten by the next step
    }
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(taddr, TMEM_COLS);
    }
}

}  // namespace bat

cudaError_t launch_vec_mod_mul_bat(const hefx_params* p, const uint32_t* x, const uint32_t* y, uint32_t* z,
                                   size_t rows, cudaStream_t s) {
    if (p->log2n < 9) return cudaErrorNotSupported;  // one limb per 512-element step
    const size_t nsteps = rows * p->n / bat::TILE;
    if (!nsteps) return cudaSuccess;
    static bool attr_set[64] = {};  // per device; benign race (idempotent)
    int dev = 0;
    cudaGetDevice(&dev);
    if (!attr_set[dev & 63]) {
        cudaError_t e = cudaFuncSetAttribute(bat::vec_mod_mul_bat_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bat::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set[dev & 63] = true;
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // 3 CTAs per SM fit in shared memory (67 KiB each); 3 x 64 TMEM columns <= 512
    const size_t grid = std::min<size_t>(nsteps, (size_t)sms * 3);
    bat::vec_mod_mul_bat_kernel<<<(unsigned)grid, bat::THREADS, bat::SMEM_BYTES, s>>>(
        p->d_lc, p->nlimbs, p->log2n, nsteps, (const uint4*)x, (const uint4*)y, (uint4*)z, p->d_err_cc);
    return cudaGetLastError();
}

}  // namespace hefx
