// Tensor-core NTT (path b), single-pass form: the layout-invariant 3-step negacyclic NTT of
// Sec. IV-B with each modular matrix product recast by BAT (Sec. IV-A, Alg. 2) as a
// low-precision matrix product on the tcgen05 tensor cores.  The NTT entry points run the
// pipelined form (ntt_tc2.cu); this one is kept for hefx_poly_mul_noalloc, whose steps
// write their results in place and need no digit workspace.
//
// Math (N = R x C, data viewed as an R x C row-major matrix; Sec. IV-B2 formula with the
// negacyclic pre-twist folded into the constants):
//   forward   B  = W1 @ A,      W1[p1][j1] = psi^(C j1 (2 brv_R(p1) + 1))
//             B' = B o T,       T[p1][j2]  = psi^(j2 (2 brv_R(p1) + 1))
//             Out = B' @ W3,    W3[j2][p2] = psi^(2R j2 brv_C(p2))
//   Out[p1][p2] is ahat at bit-reversed position p1 C + p2, i.e. the output is already in
//   the bit-reversed order (MAT's offline row/column permutations).  The inverse runs the
//   mirror: D = Ahat @ V3, D' = D o Tinv, A = V1 @ D' with N^-1 folded into V1.
//
// GB300 mapping (sm_103a has no tcgen05 int8 MMA: ptxas rejects .kind::i8 for sm_103a).
//  - Each 28-bit residue of the data is split into 4 digits of 7 bits; each constant
//    (times 2^(7i), reduced mod q -- BAT's offline fold) into 5 chunks of 6 bits.  Digits
//    and chunks are small integers held exactly in fp16, and tcgen05.mma kind::f16
//    accumulates their products in fp32: every partial sum is an integer below
//    4 * 256 * 127 * 63 < 2^23, so the accumulation is exact (bit-exact results).
//  - One GEMM per matrix step: D[(o, out)][n] = sum_k Cst[(o, out)][k] * Dig[n][k] with
//    k = (reduction index, digit).  The constant (A operand) streams through a 4-stage TMA
//    pipeline (128B swizzle); the data digits (B operand, 64 data rows x full K) are written
//    by the CUDA cores straight into the swizzled K-major layout -- the steps that reduce
//    over the data's rows get their transpose for free here.
//  - The five chunk products o of one output live in five TMEM accumulators at the same
//    lane, so an epilogue thread merges sum_o psum_o 2^(6o) in registers, reduces it with
//    one Montgomery REDC (the 2^32 factor is folded into the constants offline) and applies
//    the twiddle / Hadamard product before storing.
//  - Warp roles: warp 0 TMA producer, warp 1 MMA issuer, warp 2 TMEM owner, warps 4-7 the
//    epilogue (one TMEM lane quadrant each); all eight warps run the digit prologue.
#include <cuda.h>

#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "hefx_internal.h"
#include "host_nt.h"
#include "modarith.cuh"
#include "tc_common.cuh"

namespace hefx {

struct TcLimb {
    uint32_t q, qinv_neg, r2, pad;  // r2 = 2^64 mod q (undoes two Montgomery factors)
};

enum TcStep { FWD1 = 0, FWD3 = 1, INV1 = 2, INV3 = 3 };

struct TensorTables {
    uint32_t R = 0, C = 0;
    uint16_t* cst[4] = {nullptr, nullptr, nullptr, nullptr};  // fp16 bits [L][5][OUT][4V]
    uint2* T = nullptr;                                        // [L][R][C] forward twiddle (Shoup pairs)
    uint2* Tinv = nullptr;                                     // [L][R][C] inverse twiddle
    TcLimb* limbs = nullptr;                                   // [L]
    CUtensorMap maps[4];
    uint32_t* err = nullptr;                                   // device error flag
};

namespace {

constexpr int NT = 64;              // data rows per CTA tile (MMA N)
constexpr int STAGES = 6;           // constant pipeline depth
constexpr int KO = 5;               // 6-bit constant chunks = TMEM accumulators
constexpr uint32_t TMEM_COLS = 512;
constexpr int THREADS = 256;
constexpr uint32_t A_STAGE_BYTES = 128 * 64 * 2;  // 128 rows x 64 fp16

enum : int { OP_PLAIN = 0, OP_TW = 1, OP_HAD = 2, OP_SQUARE = 3 };

struct GemmArgs {
    const uint32_t* in;
    uint32_t* out;
    const uint32_t* had;
    const uint2* tw;  // [L][R][C] twiddle for OP_TW
    const TcLimb* limbs;
    uint32_t* err;
    uint32_t L, batch;
    uint32_t rows, cols;  // data matrix R x C
    uint32_t ntiles;      // data tiles (of NT rows of the B operand) per polynomial limb
};

size_t smem_bytes_for(uint32_t V) {
    return 1024 /*align slack*/ + (size_t)(V / 16) * NT * 128 + (size_t)STAGES * A_STAGE_BYTES + 256;
}

__device__ __forceinline__ uint32_t mont(uint32_t x, uint32_t y, uint32_t q, uint32_t qinv_neg) {
    return mul_mont_lazy(x, y, q, qinv_neg);
}

// TRANS: the GEMM reduces over the rows of the data matrix (forward step 1, inverse step 3):
//   B-operand row n = data column, k = (data row, digit); output (row, col) = (out, n).
// !TRANS: reduces over the columns (forward step 3, inverse step 1):
//   B-operand row n = data row, k = (data column, digit); output (row, col) = (n, out).
template <bool TRANS, int OP>
__global__ void __launch_bounds__(THREADS, 1) bat_ntt_gemm(const __grid_constant__ CUtensorMap cmap, GemmArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t V = TRANS ? a.rows : a.cols;  // reduction length = outputs per data row
    const uint32_t KCH = V / 16;                 // K chunks of 64 digits (4 digits per element)
    uint8_t* data_s = smem;
    uint8_t* a_s = smem + (size_t)KCH * NT * 128;
    uint64_t* full = reinterpret_cast<uint64_t*>(a_s + STAGES * A_STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* mma_done = acc_empty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);

    const uint32_t tile = blockIdx.x % a.ntiles;
    const uint32_t pl = blockIdx.x / a.ntiles;  // limb-major so co-running CTAs share constants
    const uint32_t limb = pl / a.batch, poly = pl % a.batch;
    const size_t base = ((size_t)poly * a.L + limb) * (size_t)a.rows * a.cols;
    const uint32_t n0 = tile * NT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(acc_full, 1);
        tc::mbar_init(acc_empty, 128);
        tc::mbar_init(mma_done, 1);
        tc::fence_mbar_init();
    }
    if (warp == 2) tc::tmem_alloc(tmem_slot, TMEM_COLS);
    if (threadIdx.x == 32) tc::prefetch_tmap(&cmap);

    // ---- prologue: 7-bit digits of the data tile, K-major, 128B-swizzled.  Loads are
    // issued in groups of UNR before any digit is written, to keep several in flight.
    constexpr int UNR = 8;
    if constexpr (!TRANS) {
        const uint32_t pairs = a.cols / 2;
        const uint32_t total = NT * pairs;  // multiple of THREADS * UNR for cols >= 128
        for (uint32_t t0 = threadIdx.x; t0 < total; t0 += THREADS * UNR) {
            uint2 v[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const uint32_t t = t0 + u * THREADS;
                const uint32_t rr = t / pairs, c = (t % pairs) * 2;
                v[u] = __ldg(reinterpret_cast<const uint2*>(a.in + base + (size_t)(n0 + rr) * a.cols + c));
            }
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const uint32_t t = t0 + u * THREADS;
                const uint32_t rr = t / pairs, c = (t % pairs) * 2;
                const uint2 d0 = tc::split_digits4(v[u].x), d1 = tc::split_digits4(v[u].y);
                const uint32_t k = c * 4;
                uint8_t* dst = data_s + (k >> 6) * (NT * 128) + tc::sw128_offset(rr, k & 63);
                *reinterpret_cast<uint4*>(dst) = make_uint4(d0.x, d0.y, d1.x, d1.y);
            }
        }
    } else {
        const uint32_t total = NT * (a.rows / 2);
        for (uint32_t t0 = threadIdx.x; t0 < total; t0 += THREADS * UNR) {
            uint32_t x0[UNR], x1[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const uint32_t t = t0 + u * THREADS;
                const uint32_t cc = t % NT, r = (t / NT) * 2;
                x0[u] = __ldg(a.in + base + (size_t)r * a.cols + n0 + cc);
                x1[u] = __ldg(a.in + base + (size_t)(r + 1) * a.cols + n0 + cc);
            }
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const uint32_t t = t0 + u * THREADS;
                const uint32_t cc = t % NT, r = (t / NT) * 2;
                const uint2 d0 = tc::split_digits4(x0[u]), d1 = tc::split_digits4(x1[u]);
                const uint32_t k = r * 4;
                uint8_t* dst = data_s + (k >> 6) * (NT * 128) + tc::sw128_offset(cc, k & 63);
                *reinterpret_cast<uint4*>(dst) = make_uint4(d0.x, d0.y, d1.x, d1.y);
            }
        }
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t n_ob = V / 128;  // output blocks of 128 (TMEM lanes)

    if (warp == 0) {
        if (lane == 0) {  // ---- TMA producer of constant tiles
            uint32_t stage = 0, phase = 0;
            uint32_t issued_parity[STAGES];
            bool issued[STAGES];
            for (int s = 0; s < STAGES; ++s) issued[s] = false;
            bool ok = true;
            for (uint32_t ob = 0; ob < n_ob && ok; ++ob)
                for (int o = 0; o < KO && ok; ++o)
                    for (uint32_t kc = 0; kc < KCH; ++kc) {
                        if (!tc::mbar_wait(&empty[stage], phase ^ 1u, a.err, tc::ERR_TIMEOUT_EMPTY)) {
                            ok = false;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&full[stage], A_STAGE_BYTES);
                        tc::tma_load_2d(a_s + stage * A_STAGE_BYTES, &cmap, (int32_t)(kc * 64),
                                        (int32_t)((limb * KO + o) * V + ob * 128), &full[stage]);
                        issued[stage] = true;
                        issued_parity[stage] = phase;
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
            // drain: every load this thread issued has landed before the CTA can exit
            for (int s = 0; s < STAGES; ++s)
                if (issued[s]) tc::mbar_wait(&full[s], issued_parity[s], a.err, tc::ERR_TIMEOUT_FULL);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---- MMA issuer
            const uint32_t idesc = tc::idesc_f16_f32(128, NT);
            uint32_t stage = 0, phase = 0;
            bool ok = true;
            for (uint32_t ob = 0; ob < n_ob && ok; ++ob) {
                if (ob > 0 && !tc::mbar_wait(acc_empty, (ob - 1) & 1u, a.err, tc::ERR_TIMEOUT_ACC)) break;
                tc::tc_fence_after();
                for (int o = 0; o < KO && ok; ++o)
                    for (uint32_t kc = 0; kc < KCH; ++kc) {
                        if (!tc::mbar_wait(&full[stage], phase, a.err, tc::ERR_TIMEOUT_FULL)) {
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                        const uint32_t ab = tc::smem_u32(a_s + stage * A_STAGE_BYTES);
                        const uint32_t bb = tc::smem_u32(data_s + kc * (NT * 128));
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks)
                            tc::mma_f16(tmem + o * NT, tc::sw128_desc(ab + ks * 32), tc::sw128_desc(bb + ks * 32), idesc,
                                        (kc | ks) != 0);
                        tc::mma_commit(&empty[stage]);
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                if (ok) tc::mma_commit(acc_full);
            }
            // every MMA this thread issued has completed before TMEM is released
            tc::mma_commit(mma_done);
            tc::mbar_wait(mma_done, 0, a.err, tc::ERR_TIMEOUT_ACC);
        }
    } else if (warp >= 4) {  // ---- epilogue: one TMEM lane quadrant per warp
        const uint32_t lq = (uint32_t)(warp - 4) * 32;
        const TcLimb lc = a.limbs[limb];
        for (uint32_t ob = 0; ob < n_ob; ++ob) {
            if (!tc::mbar_wait(acc_full, ob & 1u, a.err, tc::ERR_TIMEOUT_ACC)) break;
            tc::tc_fence_after();
            const uint32_t outi = ob * 128 + lq + lane;  // output index held by this thread
            for (int cb = 0; cb < NT; cb += 16) {
                uint32_t acc[KO][16];
#pragma unroll
                for (int o = 0; o < KO; ++o) tc::tmem_ld16(tmem + (lq << 16) + o * NT + cb, acc[o]);
                tc::tmem_ld_wait();
                uint32_t res[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const uint64_t z = (uint64_t)tc::acc_to_u32(acc[0][j]) + ((uint64_t)tc::acc_to_u32(acc[1][j]) << 6) +
                                       ((uint64_t)tc::acc_to_u32(acc[2][j]) << 12) +
                                       ((uint64_t)tc::acc_to_u32(acc[3][j]) << 18) +
                                       ((uint64_t)tc::acc_to_u32(acc[4][j]) << 24);
                    // Montgomery REDC: z 2^-32 mod q in [0, 2q) (z < 2^48 < q 2^32)
                    const uint32_t zl = (uint32_t)z, zh = (uint32_t)(z >> 32);
                    uint32_t r = zh + __umulhi(zl * lc.qinv_neg, lc.q) + (zl != 0u);
                    const uint32_t n = n0 + cb + j;
                    const uint32_t row = TRANS ? outi : n, col = TRANS ? n : outi;
                    const size_t pos = (size_t)row * a.cols + col;
                    if constexpr (OP == OP_TW) {
                        const uint2 w = __ldg(a.tw + (size_t)limb * a.rows * a.cols + pos);
                        r = mul_shoup_lazy(r, w.x, w.y, lc.q);
                    } else if constexpr (OP == OP_HAD) {
                        const uint32_t h = __ldg(a.had + base + pos);
                        r = mont(mont(r, h, lc.q, lc.qinv_neg), lc.r2, lc.q, lc.qinv_neg);
                    } else if constexpr (OP == OP_SQUARE) {
                        const uint32_t rc = csub(r, lc.q);
                        r = mont(mont(rc, rc, lc.q, lc.qinv_neg), lc.r2, lc.q, lc.qinv_neg);
                    }
                    res[j] = csub(r, lc.q);
                }
                if constexpr (TRANS) {
                    uint4* dst = reinterpret_cast<uint4*>(a.out + base + (size_t)outi * a.cols + n0 + cb);
#pragma unroll
                    for (int j = 0; j < 16; j += 4) dst[j / 4] = make_uint4(res[j], res[j + 1], res[j + 2], res[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) a.out[base + (size_t)(n0 + cb + j) * a.cols + outi] = res[j];
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(acc_empty);
        }
    }
    __syncthreads();
    if (warp == 2) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// ------------------------------------------------------------------ host tables

uint16_t half_bits_small(uint32_t d) {  // exact fp16 of an integer 0 <= d < 2048
    if (d == 0) return 0;
    int e = 31 - __builtin_clz(d);
    return (uint16_t)(((e + 15) << 10) | ((d << (10 - e)) & 0x3FFu));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) == cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

bool encode_map_2d(CUtensorMap* map, CUtensorMapDataType dtype, void* base, uint64_t inner, uint64_t rows,
                   uint64_t row_bytes, uint32_t box_inner, uint32_t box_rows, CUtensorMapSwizzle swz) {
    if (!encode_fn()) return false;
    const cuuint64_t dims[2] = {inner, rows};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {box_inner, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode_fn()(map, dtype, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_supported(const hefx_params* p) {
    // 8-bit digits (moduli above 2^28) need every factor <= 64: no split of 2^13 has that
    return p->log2n >= 12 && p->log2n <= 16 && encode_fn() && !(tc2_wide(p) && p->log2n == 13);
}

bool tc_narrow(const hefx_params* p) {
    // the single-pass form: N = 2^14 .. 2^16, 6-bit chunks of 28-bit moduli
    return tc_supported(p) && p->log2n >= 14 && p->max_prime < (1u << 28);
}

void tc_free(hefx_params* p) {
    tc2_free(p);
    TensorTables* t = p->tc;
    if (!t) return;
    for (int i = 0; i < 4; ++i)
        if (t->cst[i]) cudaFree(t->cst[i]);
    if (t->T) cudaFree(t->T);
    if (t->Tinv) cudaFree(t->Tinv);
    if (t->limbs) cudaFree(t->limbs);
    if (t->err) cudaFree(t->err);
    delete t;
    p->tc = nullptr;
}

// Offline precompute (Sec. IV-A "compile time"): W1, T, W3 and their inverses per limb,
// then OfflineCompileLeft of Alg. 2 with 7-bit input digits and 6-bit output chunks, all
// constants multiplied by 2^32 so the epilogue's Montgomery REDC returns the plain value.
cudaError_t tc_prepare(hefx_params* p) {
    if (!encode_fn()) return cudaErrorNotSupported;
    const uint32_t logn = p->log2n, N = p->n, L = p->nlimbs;
    const uint32_t logR = logn / 2, R = 1u << logR, C = N / R, logC = logn - logR;
    TensorTables* t = new TensorTables();
    t->R = R;
    t->C = C;
    const uint32_t outs[4] = {R, C, C, R}, Vs[4] = {R, C, C, R};
    std::vector<std::vector<uint16_t>> hc(4);
    for (int s = 0; s < 4; ++s) hc[s].assign((size_t)L * KO * outs[s] * 4 * Vs[s], 0);
    std::vector<uint2> hT((size_t)L * N), hTi((size_t)L * N);
    std::vector<TcLimb> hl(L);

    auto work = [&](uint32_t l) {
        const uint64_t q = p->primes[l], psi = p->psi[l], twoN = 2ull * N;
        std::vector<uint64_t> pw(twoN);
        pw[0] = 1;
        for (uint64_t e = 1; e < twoN; ++e) pw[e] = mul_mod(pw[e - 1], psi, q);
        auto P = [&](uint64_t e) { return pw[e % twoN]; };
        auto Pn = [&](uint64_t e) { return pw[(twoN - e % twoN) % twoN]; };
        const uint64_t r32 = ((uint64_t)1 << 32) % q, ninv = inv_mod(N % q, q);
        hl[l].q = (uint32_t)q;
        hl[l].qinv_neg = neg_inv_pow2_32((uint32_t)q);
        hl[l].r2 = (uint32_t)mul_mod(r32, r32, q);
        hl[l].pad = 0;
        // BAT block of constant w at (out, v) of step s: chunk_o((w 2^32) 2^(7i) mod q)
        auto put = [&](int s, uint32_t out, uint32_t v, uint64_t w) {
            const uint32_t OUTs = outs[s], K = 4 * Vs[s];
            uint64_t c = mul_mod(w, r32, q);
            for (uint32_t i = 0; i < 4; ++i) {
                for (int o = 0; o < KO; ++o) {
                    const uint32_t chunk = (uint32_t)((c >> (6 * o)) & 63u);
                    hc[s][(((size_t)l * KO + o) * OUTs + out) * K + v * 4 + i] = half_bits_small(chunk);
                }
                c = (c << 7) % q;
            }
        };
        for (uint32_t p1 = 0; p1 < R; ++p1) {
            const uint64_t kodd = 2ull * bit_reverse(p1, (int)logR) + 1;
            for (uint32_t j1 = 0; j1 < R; ++j1) {
                put(FWD1, p1, j1, P((uint64_t)C * j1 * kodd));                      // W1[p1][j1]
                put(INV3, j1, p1, mul_mod(ninv, Pn((uint64_t)C * j1 * kodd), q));   // V1[j1][p1]
            }
            for (uint32_t j2 = 0; j2 < C; ++j2) {
                const uint64_t w = P((uint64_t)j2 * kodd), wi = Pn((uint64_t)j2 * kodd);
                hT[(size_t)l * N + (size_t)p1 * C + j2] = make_uint2((uint32_t)w, shoup(w, q));
                hTi[(size_t)l * N + (size_t)p1 * C + j2] = make_uint2((uint32_t)wi, shoup(wi, q));
            }
        }
        for (uint32_t p2 = 0; p2 < C; ++p2) {
            const uint64_t kb = bit_reverse(p2, (int)logC);
            for (uint32_t j2 = 0; j2 < C; ++j2) {
                put(FWD3, p2, j2, P(2ull * R * j2 * kb));   // W3[j2][p2]
                put(INV1, j2, p2, Pn(2ull * R * j2 * kb));  // V3[p2][j2]
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
    for (int s = 0; s < 4 && e == cudaSuccess; ++s) {
        e = cudaMalloc(&t->cst[s], hc[s].size() * 2);
        if (e == cudaSuccess) e = cudaMemcpy(t->cst[s], hc[s].data(), hc[s].size() * 2, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&t->T, hT.size() * sizeof(uint2));
    if (e == cudaSuccess) e = cudaMemcpy(t->T, hT.data(), hT.size() * sizeof(uint2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&t->Tinv, hTi.size() * sizeof(uint2));
    if (e == cudaSuccess) e = cudaMemcpy(t->Tinv, hTi.data(), hTi.size() * sizeof(uint2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&t->limbs, L * sizeof(TcLimb));
    if (e == cudaSuccess) e = cudaMemcpy(t->limbs, hl.data(), L * sizeof(TcLimb), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&t->err, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(t->err, 0, sizeof(uint32_t));
    for (int s = 0; s < 4 && e == cudaSuccess; ++s) {
        const cuuint64_t K = 4ull * Vs[s];
        const cuuint64_t dims[2] = {K, (cuuint64_t)L * KO * outs[s]};
        const cuuint64_t strides[1] = {K * 2};
        const cuuint32_t box[2] = {64, 128};
        const cuuint32_t estr[2] = {1, 1};
        CUresult r = encode_fn()(&t->maps[s], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, t->cst[s], dims, strides, box, estr,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) {
        p->tc = t;
        tc_free(p);
        return e;
    }
    p->tc = t;
    return cudaSuccess;
}

namespace {

template <bool TRANS, int OP>
cudaError_t launch_gemm(const CUtensorMap& map, const GemmArgs& g, uint32_t V, cudaStream_t s) {
    auto kern = bat_ntt_gemm<TRANS, OP>;
    const size_t smem = smem_bytes_for(V);
    static size_t attr_bytes = 0;  // per instantiation; idempotent
    if (attr_bytes < smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_bytes = smem;
    }
    const uint32_t grid = g.L * g.batch * g.ntiles;
    kern<<<grid, THREADS, smem, s>>>(map, g);
    return cudaGetLastError();
}

// One matrix step over the whole batch.
cudaError_t run_step(const hefx_params* p, TcStep step, int op, const uint32_t* in, const uint32_t* had,
                     uint32_t* out, size_t batch, cudaStream_t s) {
    const TensorTables* t = p->tc;
    GemmArgs g;
    g.in = in;
    g.out = out;
    g.had = had;
    g.tw = (step == FWD1) ? t->T : t->Tinv;
    g.limbs = t->limbs;
    g.err = t->err;
    g.L = p->nlimbs;
    g.batch = (uint32_t)batch;
    g.rows = t->R;
    g.cols = t->C;
    const bool trans = (step == FWD1 || step == INV3);
    const uint32_t V = trans ? t->R : t->C;        // reduction length
    const uint32_t DN = trans ? t->C : t->R;       // data rows of the B operand
    g.ntiles = DN / NT;
    const CUtensorMap& m = t->maps[step];
    if (trans) {
        if (op == OP_TW) return launch_gemm<true, OP_TW>(m, g, V, s);
        return launch_gemm<true, OP_PLAIN>(m, g, V, s);
    }
    switch (op) {
        case OP_TW: return launch_gemm<false, OP_TW>(m, g, V, s);
        case OP_HAD: return launch_gemm<false, OP_HAD>(m, g, V, s);
        case OP_SQUARE: return launch_gemm<false, OP_SQUARE>(m, g, V, s);
        default: return launch_gemm<false, OP_PLAIN>(m, g, V, s);
    }
}

}  // namespace

// ------------------------------------------------------------------ no-allocation product
// Workspace of hefx_poly_mul_noalloc: a fixed device array in the library image, so that
// call never allocates.  Every device that loads the library holds these bytes until the
// process exits; every call on a device shares them.
constexpr size_t kNoallocScratchWords = (size_t)1 << 21;  // 8 MiB
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoallocScratchWords];

namespace {
// Device address of g_noalloc_scratch per device ordinal, looked up once with that device
// current (the host-side name is only a stand-in for the symbol, not a device address).
std::mutex g_noalloc_mu;
uint32_t* g_noalloc_ptr[128] = {};
}  // namespace

size_t noalloc_scratch_words() { return kNoallocScratchWords; }

cudaError_t polymul_tc_noalloc(const hefx_params* p, const uint32_t* a, const uint32_t* b, uint32_t* c, size_t batch,
                               cudaStream_t s) {
    if (batch == 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    uint32_t* S;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) return e;
            g_noalloc_ptr[dev] = static_cast<uint32_t*>(ptr);
        }
        S = g_noalloc_ptr[dev];
    }
    // the step sequence of the tensor-path product, with the static array as the workspace;
    // S is fully written (forward step 1) before it is read, so nothing needs clearing
    if (a == b) {
        e = run_step(p, FWD1, OP_TW, a, nullptr, S, batch, s);
        if (e == cudaSuccess) e = run_step(p, FWD3, OP_SQUARE, S, nullptr, c, batch, s);
    } else {
        if (c == b) std::swap(a, b);
        e = run_step(p, FWD1, OP_TW, a, nullptr, c, batch, s);
        if (e == cudaSuccess) e = run_step(p, FWD3, OP_PLAIN, c, nullptr, c, batch, s);
        if (e == cudaSuccess) e = run_step(p, FWD1, OP_TW, b, nullptr, S, batch, s);
        if (e == cudaSuccess) e = run_step(p, FWD3, OP_HAD, S, c, c, batch, s);
    }
    if (e == cudaSuccess) e = run_step(p, INV1, OP_TW, c, nullptr, c, batch, s);
    if (e == cudaSuccess) e = run_step(p, INV3, OP_PLAIN, c, nullptr, c, batch, s);
    return e;
}

// Reads and clears the device error flag of the tensor path (synchronizes the stream).
cudaError_t tc_check(const hefx_params* p, cudaStream_t s, uint32_t* code) {
    *code = 0;
    if (!p->tc) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(code, p->tc->err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && *code) e = cudaMemsetAsync(p->tc->err, 0, 4, s);
    return e;
}

}  // namespace hefx
