// Tensor-core basis conversion (path c): App. B's BConv with its step-2 MatModMul turned
// into a BAT digit-split matrix product (Sec. IV-A3, "High-Precision MatModMul in BConv").
//
//   D[n][(j, o)] = sum_{(i, d)} digit_d(b_{n,i}) * chunk_o([qhat_i]_{p_j} 2^32 2^(7d) mod p_j)
//   out_{n,j}    = REDC_{p_j}( sum_o D[n][(j, o)] 2^(8o) )
//
// b_{n,i} = [a_{n,i} qhat_i^-1]_{q_i} is step 1 (a Shoup product in the prologue); digits are
// 7 bits (b < q_i < 2^28), chunks 8 bits (four per constant < p_j < 2^32; integers up to 2048
// are exact in fp16), and every partial sum is below 4 * 64 * 127 * 255 < 2^23, so fp16
// operands with fp32 accumulation are exact.  Four chunk columns per target limb put up to
// 64 targets in one 256-column MMA (N = 256), two accumulators in 512 TMEM columns.
//
// GB300 mapping: a persistent kernel streams 128-coefficient tiles.  One thread keeps four
// raw residue tiles (L rows x 128 coefficients) in flight with TMA; four producer warps apply
// step 1 to a staged tile and write the digits into a double-buffered K-major 128B-swizzled
// A tile; one thread issues the tcgen05 MMAs against
// the constant B operand (resident in shared memory for the whole kernel) into one of two
// TMEM accumulators; four epilogue warps merge, reduce mod p_j and store while the next tile
// is being produced.  The operation is HBM-bound (16 B per source residue in, 4 per
// target residue out per coefficient), so the tensor pipe is mostly idle by design.
#include <cstring>
#include <vector>

#include "bconv_common.h"
#include "host_nt.h"
#include "modarith.cuh"
#include "tc_common.cuh"

namespace hefx {

namespace {

constexpr int KO = 4;
#ifndef HEFX_BC_NPG
#define HEFX_BC_NPG 2
#endif
constexpr int NPG = HEFX_BC_NPG;  // producer groups of 4 warps (each takes every NPG-th source limb)
// warps 0-3 and 8-11 producer groups 0 and 1, 4-7 epilogue, 12 MMA, 13 TMA, 14.. further producer groups
constexpr int THREADS = (14 + 4 * (NPG - 2)) * 32;
constexpr int MAX_L = 48, MAX_LP = 64;  // MAX_L: 4 staged raw tiles fit in shared memory; MAX_LP: MMA N <= 256

struct BcTcConst {
    uint32_t L, Lp, kpad, npad;      // K = 4L padded to 64, N = 4 columns per target limb, padded to 16
    uint32_t q[MAX_L], qhat_inv[MAX_L], qhat_inv_sh[MAX_L];
    uint32_t p[MAX_LP], pinv_neg[MAX_LP];
};

struct BcTcPlan {
    BcTcConst* d_const = nullptr;
    uint8_t* d_bimage = nullptr;  // constant B operand, already in the swizzled smem layout
    uint32_t bimage_bytes = 0;
    uint32_t kpad = 0, npad = 0, tmem_cols = 0;
};

uint16_t half_bits_small(uint32_t d) {
    if (d == 0) return 0;
    int e = 31 - __builtin_clz(d);
    return (uint16_t)(((e + 15) << 10) | ((d << (10 - e)) & 0x3FFu));
}

uint32_t sw128_offset_host(uint32_t row, uint32_t k) {
    const uint32_t chunk = (k >> 3) & 7u;
    return row * 128u + ((chunk ^ (row & 7u)) << 4) + ((k & 7u) << 1);
}

constexpr int RAW_STAGES = 4;

// raw residue tile: L rows (source limbs) x 128 coefficients, uint32, dense
size_t raw_bytes(uint32_t L) { return (size_t)L * 128 * 4; }

size_t smem_bytes(const BcTcPlan& tp, uint32_t L) {
    return 1024 + 2ull * 128 * tp.kpad * 2 + tp.bimage_bytes + RAW_STAGES * raw_bytes(L) + 256;
}

// Warp roles: 0-3 and 8-11 producers (step 1 + digits; the two groups split the source limbs
// of a tile), 4-7 epilogue, 12 MMA issuer + TMEM owner, 13 TMA issuer of raw residue tiles.
__global__ void __launch_bounds__(THREADS, 1)
    bconv_tc_kernel(const __grid_constant__ CUtensorMap in_map, const BcTcConst* __restrict__ gc,
                    const uint8_t* __restrict__ bimage, uint32_t bimage_bytes, uint32_t* __restrict__ out, uint32_t n,
                    uint32_t batch, uint32_t tmem_cols, uint32_t* err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ BcTcConst c;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (uint32_t i = tid; i < sizeof(BcTcConst) / 4; i += THREADS)
        reinterpret_cast<uint32_t*>(&c)[i] = reinterpret_cast<const uint32_t*>(gc)[i];
    const uint32_t kpad0 = gc->kpad, L0 = gc->L;
    const uint32_t abytes = 128 * kpad0 * 2;  // one A tile: 128 rows x K fp16
    const uint32_t rbytes = L0 * 128 * 4;
    uint8_t* a_s[2] = {smem, smem + abytes};
    uint8_t* b_s = smem + 2 * abytes;
    uint8_t* raw_s = b_s + bimage_bytes;  // RAW_STAGES x rbytes (16-byte aligned)
    uint64_t* bars = reinterpret_cast<uint64_t*>(raw_s + RAW_STAGES * rbytes);
    uint64_t* a_full = bars;        // [2] producer -> MMA
    uint64_t* a_empty = bars + 2;   // [2] MMA -> producer
    uint64_t* acc_full = bars + 4;  // [2] MMA -> epilogue
    uint64_t* acc_empty = bars + 6; // [2] epilogue -> MMA
    uint64_t* mma_done = bars + 8;
    uint64_t* raw_full = bars + 9;                // [RAW_STAGES] TMA -> producer
    uint64_t* raw_empty = raw_full + RAW_STAGES;  // [RAW_STAGES] producer -> TMA
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(raw_empty + RAW_STAGES);

    // constant B operand and zeroed A tiles (K padding stays zero for the whole kernel)
    for (uint32_t i = tid; i < bimage_bytes / 16; i += THREADS)
        reinterpret_cast<uint4*>(b_s)[i] = reinterpret_cast<const uint4*>(bimage)[i];
    for (uint32_t i = tid; i < 2 * abytes / 16; i += THREADS) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&a_full[s], 128 * NPG);
            tc::mbar_init(&a_empty[s], 1);
            tc::mbar_init(&acc_full[s], 1);
            tc::mbar_init(&acc_empty[s], 128);
        }
        for (int s = 0; s < RAW_STAGES; ++s) {
            tc::mbar_init(&raw_full[s], 1);
            tc::mbar_init(&raw_empty[s], 128 * NPG);
        }
        tc::mbar_init(mma_done, 1);
        tc::fence_mbar_init();
    }
    if (warp == 12) tc::tmem_alloc(tmem_slot, tmem_cols);
    if (tid == 13 * 32) tc::prefetch_tmap(&in_map);
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t L = c.L, Lp = c.Lp, npad = c.npad;
    const uint32_t tiles_per_poly = n / 128;
    const uint32_t ntiles = tiles_per_poly * batch;

    if (warp == 13) {  // ---- TMA issuer: raw residue tiles, RAW_STAGES in flight
        if (lane == 0) {
            uint32_t it = 0;
            bool issued[RAW_STAGES];
            uint32_t par[RAW_STAGES];
            for (int s = 0; s < RAW_STAGES; ++s) issued[s] = false;
            for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
                const uint32_t s = it % RAW_STAGES, ph = (it / RAW_STAGES) & 1;
                if (!tc::mbar_wait(&raw_empty[s], ph ^ 1u, err, tc::ERR_TIMEOUT_EMPTY)) break;
                const uint32_t b = t / tiles_per_poly, x0 = (t % tiles_per_poly) * 128;
                tc::mbar_arrive_expect_tx(&raw_full[s], rbytes);
                tc::tma_load_2d(raw_s + s * rbytes, &in_map, (int32_t)x0, (int32_t)(b * L), &raw_full[s]);
                issued[s] = true;
                par[s] = ph;
            }
            for (int s = 0; s < RAW_STAGES; ++s)
                if (issued[s]) tc::mbar_wait(&raw_full[s], par[s], err, tc::ERR_TIMEOUT_FULL);
        }
    } else if (warp < 4 || (warp >= 8 && warp < 12) || warp >= 14) {  // ---- producers: step 1 and digit split
        // coefficient row, and the group (source limbs i = grp mod NPG)
        const uint32_t row = tid & 127, grp = warp < 4 ? 0u : warp < 12 ? 1u : 2u + (warp - 14) / 4;
        uint32_t it = 0;
        for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const uint32_t s = it & 1, ph = (it >> 1) & 1;
            const uint32_t rs = it % RAW_STAGES, rph = (it / RAW_STAGES) & 1;
            if (!tc::mbar_wait(&raw_full[rs], rph, err, tc::ERR_TIMEOUT_FULL)) break;
            if (!tc::mbar_wait(&a_empty[s], ph ^ 1u, err, tc::ERR_TIMEOUT_EMPTY)) break;
            const uint32_t* raw = reinterpret_cast<const uint32_t*>(raw_s + rs * rbytes) + row;
            uint8_t* A = a_s[s];
            for (uint32_t i = grp; i < L; i += NPG) {
                const uint32_t qi = c.q[i];
                const uint32_t bi = csub(mul_shoup_lazy(raw[i * 128], c.qhat_inv[i], c.qhat_inv_sh[i], qi), qi);
                const uint2 d = tc::split_digits4(bi);
                const uint32_t k = 4 * i;
                *reinterpret_cast<uint2*>(A + (k >> 6) * (128 * 128) + tc::sw128_offset(row, k & 63)) = d;
            }
            tc::mbar_arrive(&raw_empty[rs]);
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&a_full[s]);
        }
    } else if (warp >= 4 && warp < 8) {  // ---- epilogue: merge, reduce mod p_j, store
        const uint32_t lq = (warp - 4) * 32;
        uint32_t it = 0;
        for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const uint32_t s = it & 1, ph = (it >> 1) & 1;
            if (!tc::mbar_wait(&acc_full[s], ph, err, tc::ERR_TIMEOUT_ACC)) break;
            tc::tc_fence_after();
            const uint32_t b = t / tiles_per_poly, x = (t % tiles_per_poly) * 128 + lq + lane;
            uint32_t* dst = out + (size_t)b * Lp * n + x;
            // columns: output j's four chunk sums sit at 4j .. 4j+3, four outputs per 16 columns
            for (uint32_t cb = 0; cb < npad; cb += 16) {
                uint32_t r[16];
                tc::tmem_ld16(tmem + (lq << 16) + s * npad + cb, r);
                tc::tmem_ld_wait();
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const uint32_t j = cb / 4 + h;
                    if (j < Lp) {
                        const uint64_t z = (uint64_t)tc::acc_to_u32(r[4 * h]) +
                                           ((uint64_t)tc::acc_to_u32(r[4 * h + 1]) << 8) +
                                           ((uint64_t)tc::acc_to_u32(r[4 * h + 2]) << 16) +
                                           ((uint64_t)tc::acc_to_u32(r[4 * h + 3]) << 24);
                        const uint32_t pj = c.p[j];
                        const uint32_t zl = (uint32_t)z, zh = (uint32_t)(z >> 32);
                        const uint32_t rr = zh + __umulhi(zl * c.pinv_neg[j], pj) + (zl != 0u);
                        dst[(size_t)j * n] = csub(rr, pj);
                    }
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&acc_empty[s]);
        }
    } else if (warp == 12 && lane == 0) {  // ---- MMA issuer
        const uint32_t idesc = tc::idesc_f16_f32(128, npad);
        const uint32_t ksteps = (4 * L + 15) / 16;
        uint32_t it = 0;
        for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const uint32_t s = it & 1, ph = (it >> 1) & 1;
            if (!tc::mbar_wait(&a_full[s], ph, err, tc::ERR_TIMEOUT_FULL)) break;
            if (!tc::mbar_wait(&acc_empty[s], ph ^ 1u, err, tc::ERR_TIMEOUT_ACC)) break;
            tc::tc_fence_after();
            for (uint32_t ks = 0; ks < ksteps; ++ks) {
                const uint32_t kc = ks >> 2, kin = ks & 3;
                const uint32_t ab = tc::smem_u32(a_s[s] + kc * (128 * 128)) + kin * 32;
                const uint32_t bb = tc::smem_u32(b_s + kc * (npad * 128)) + kin * 32;
                tc::mma_f16(tmem + s * npad, tc::sw128_desc(ab), tc::sw128_desc(bb), idesc, ks != 0);
            }
            tc::mma_commit(&acc_full[s]);
            tc::mma_commit(&a_empty[s]);
        }
        tc::mma_commit(mma_done);
        tc::mbar_wait(mma_done, 0, err, tc::ERR_TIMEOUT_ACC);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 12) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, tmem_cols);
    }
}

}  // namespace

bool bconv_tc_available(const hefx_bconv_plan* plan) {
    return plan->d_bat != nullptr && plan->log2n >= 7;
}

bool bconv_prefer_tc(const hefx_bconv_plan* plan, size_t batch) {
    // measured at N = 2^16: the tensor kernel wins only where many targets share each source
    // digit (24 -> 56 at batch 8: 132 vs 138 us); 8 to 40 targets and small calls favour the
    // CUDA-core kernel (24 -> 8: 76 vs 54 us, 16 -> 40 at batch 8: 97 vs 81 us)
    return bconv_tc_available(plan) && plan->Lp >= 48 && ((batch * plan->L) << plan->log2n) >= ((size_t)96 << 16);
}

// Offline compile of the step-2 constant (OfflineCompileLeft of Alg. 2 for the right-hand
// constant matrix): row (j, o), column (i, d) holds chunk_o([qhat_i]_{p_j} 2^32 2^(7d) mod p_j),
// laid out exactly as the kernel's shared-memory B tile (K-major, 128B swizzle).
cudaError_t bconv_tc_upload(hefx_bconv_plan* plan, const BConvConst& h) {
    const uint32_t L = plan->L, Lp = plan->Lp;
    for (uint32_t i = 0; i < L; ++i)
        if (plan->src[i] >= (1u << 28)) return cudaSuccess;  // digits need 28-bit sources
    if (L > (uint32_t)MAX_L || Lp > (uint32_t)MAX_LP) return cudaSuccess;  // CUDA-core path only
    BcTcPlan* tp = new BcTcPlan();
    tp->kpad = ((4 * L + 63) / 64) * 64;
    tp->npad = ((KO * Lp + 15) / 16) * 16;
    uint32_t cols = 32;
    while (cols < 2 * tp->npad) cols *= 2;
    tp->tmem_cols = cols;
    tp->bimage_bytes = tp->npad * tp->kpad * 2;
    if (smem_bytes(*tp, L) > 232448) {  // does not fit one CTA's shared memory: CUDA-core path only
        delete tp;
        return cudaSuccess;
    }
    std::vector<uint8_t> img(tp->bimage_bytes, 0);
    for (uint32_t j = 0; j < Lp; ++j) {
        const uint64_t p = plan->dst[j];
        const uint64_t r32 = ((uint64_t)1 << 32) % p;
        for (uint32_t i = 0; i < L; ++i) {
            uint64_t cst = mul_mod(h.qhat_p[i * kBConvMaxLimbs + j], r32, p);
            for (uint32_t d = 0; d < 4; ++d) {
                const uint32_t k = 4 * i + d;
                for (int o = 0; o < KO; ++o) {
                    const uint32_t row = KO * j + o;
                    const uint16_t hb = half_bits_small((uint32_t)((cst >> (8 * o)) & 255u));
                    const size_t off = (size_t)(k / 64) * (tp->npad * 128) + sw128_offset_host(row, k % 64);
                    memcpy(&img[off], &hb, 2);
                }
                cst = (cst << 7) % p;
            }
        }
    }
    BcTcConst hc;
    memset(&hc, 0, sizeof hc);
    hc.L = L;
    hc.Lp = Lp;
    hc.kpad = tp->kpad;
    hc.npad = tp->npad;
    for (uint32_t i = 0; i < L; ++i) {
        hc.q[i] = h.q[i];
        hc.qhat_inv[i] = h.qhat_inv[i];
        hc.qhat_inv_sh[i] = h.qhat_inv_sh[i];
    }
    for (uint32_t j = 0; j < Lp; ++j) {
        hc.p[j] = h.p[j];
        hc.pinv_neg[j] = neg_inv_pow2_32(h.p[j]);
    }
    cudaError_t e = cudaMalloc(&tp->d_const, sizeof hc);
    if (e == cudaSuccess) e = cudaMemcpy(tp->d_const, &hc, sizeof hc, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&tp->d_bimage, img.size());
    if (e == cudaSuccess) e = cudaMemcpy(tp->d_bimage, img.data(), img.size(), cudaMemcpyHostToDevice);
    plan->d_bat = tp;
    if (e != cudaSuccess) {
        bconv_tc_free(plan);
        return e;
    }
    return cudaSuccess;
}

void bconv_tc_free(hefx_bconv_plan* plan) {
    BcTcPlan* tp = static_cast<BcTcPlan*>(plan->d_bat);
    if (!tp) return;
    if (tp->d_const) cudaFree(tp->d_const);
    if (tp->d_bimage) cudaFree(tp->d_bimage);
    delete tp;
    plan->d_bat = nullptr;
}

cudaError_t launch_bconv_tc(const hefx_bconv_plan* plan, const uint32_t* in, uint32_t* out, size_t batch,
                            cudaStream_t stream) {
    const BcTcPlan* tp = static_cast<const BcTcPlan*>(plan->d_bat);
    if (!tp || plan->log2n < 7) return cudaErrorNotSupported;
    const uint32_t n = 1u << plan->log2n;
    const size_t ntiles = (size_t)(n / 128) * batch;
    if (ntiles == 0) return cudaSuccess;
    // raw residues of the batch as a 2D array: rows (b, i) of n coefficients
    CUtensorMap in_map;
    if (!encode_map_2d(&in_map, CU_TENSOR_MAP_DATA_TYPE_UINT32, const_cast<uint32_t*>(in), n, batch * plan->L,
                       (uint64_t)n * 4, 128, plan->L, CU_TENSOR_MAP_SWIZZLE_NONE))
        return cudaErrorInvalidValue;
    const size_t smem = smem_bytes(*tp, plan->L);
    static size_t attr = 0;
    if (attr < smem) {
        cudaError_t e = cudaFuncSetAttribute(bconv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)std::min<size_t>(ntiles, (size_t)sms);
    bconv_tc_kernel<<<grid, THREADS, smem, stream>>>(in_map, tp->d_const, tp->d_bimage, tp->bimage_bytes, out, n,
                                                      (uint32_t)batch, tp->tmem_cols, plan->d_err);
    return cudaGetLastError();
}

}  // namespace hefx
