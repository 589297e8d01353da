// RNS basis conversion (App. B, BConv), CUDA-core path and plan constants.
//
//   out_{n,j} = sum_i [a_{n,i} * qhat_i^-1]_{q_i} * [qhat_i]_{p_j}  mod p_j
//
// The same kernel with a ModDown epilogue finishes hybrid key switching (the HE-Mult of
// Sec. V-A): with the plan's sources the special primes P and its targets the ciphertext
// primes, out_{n,j} = (x_{n,j} - BConv(x_P)_{n,j}) * P^-1 mod q_j.  Its exact variant
// subtracts v Q with v = round(sum_i b_i / q_i), estimated as a 128-bit fixed-point sum
// sum_i b_i round(2^k / q_i) (error below 2^-55 Q), which yields the centered CRT value
// mod p_j (the u-corrected conversion; the paper prints only the fast one).
//
// Step 1 is L independent VecModMuls by the constant qhat_i^-1 (Shoup products); step 2
// is an (N, L, L') MatModMul whose right operand is the constant matrix [qhat_i]_{p_j}.
// This file runs step 2 as 64-bit multiply-accumulates (each product < 2^58, L <= 64
// products fit in 64 bits) with one Barrett reduction per output; bconv_tc.cu runs it on
// the tensor cores as a digit-split (BAT) matrix product.
#include <algorithm>
#include <vector>

#include "bconv_common.h"
#include "host_nt.h"
#include "modarith.cuh"

namespace hefx {

void fill_bconv_const(const uint32_t* src, uint32_t L, const uint32_t* dst, uint32_t Lp, BConvConst& h) {
    memset(&h, 0, sizeof(h));
    h.L = L;
    h.Lp = Lp;
    for (uint32_t i = 0; i < L; ++i) {
        const uint64_t q = src[i];
        uint64_t qhat = 1;
        for (uint32_t k = 0; k < L; ++k)
            if (k != i) qhat = mul_mod(qhat, src[k], q);
        const uint64_t qi = inv_mod(qhat, q);
        h.q[i] = (uint32_t)q;
        h.qhat_inv[i] = (uint32_t)qi;
        h.qhat_inv_sh[i] = shoup(qi, q);
        h.qpack[i][0] = h.q[i];
        h.qpack[i][1] = h.qhat_inv[i];
        h.qpack[i][2] = h.qhat_inv_sh[i];
        for (uint32_t j = 0; j < Lp; ++j) {
            uint64_t c = 1;
            for (uint32_t k = 0; k < L; ++k)
                if (k != i) c = mul_mod(c, src[k], dst[j]);
            h.qhat_p[i * kBConvMaxLimbs + j] = (uint32_t)c;
        }
    }
    for (uint32_t j = 0; j < Lp; ++j) {
        h.p[j] = dst[j];
        h.p_mu[j] = (uint64_t)(((u128)1 << 64) / dst[j]);  // floor(2^64 / p_j)
        uint64_t prod = 1;
        for (uint32_t i = 0; i < L; ++i) prod = mul_mod(prod, src[i], dst[j]);
        const uint64_t pinv = inv_mod(prod, dst[j]);
        h.pinv[j] = (uint32_t)pinv;
        h.pinv_sh[j] = shoup(pinv, dst[j]);
        h.qmod_p[j] = (uint32_t)prod;
    }
    // exact conversion: k = 63 + floor(log2(min q_i)) keeps every w_i = round(2^k / q_i) below 2^64
    uint32_t minq = src[0];
    for (uint32_t i = 1; i < L; ++i) minq = std::min(minq, src[i]);
    int lg = 0;
    while ((2u << lg) <= minq) ++lg;
    const int k = 63 + lg;
    for (uint32_t i = 0; i < L; ++i) {
        const u128 num = (u128)1 << k;
        const u128 qi = src[i];
        h.w[i] = (uint64_t)((num + qi / 2) / qi);
    }
    const u128 half = (u128)1 << (k - 1);
    h.half_lo = (uint64_t)half;
    h.half_hi = (uint64_t)(half >> 64);
    h.kshift = (uint32_t)(k - 64);
}

cudaError_t bconv_plan_upload(hefx_bconv_plan* plan) {
    BConvConst h;
    fill_bconv_const(plan->src.data(), plan->L, plan->dst.data(), plan->Lp, h);
    cudaError_t e = cudaMalloc(&plan->d_const, sizeof(BConvConst));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(plan->d_const, &h, sizeof(BConvConst), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&plan->d_err, 4);
    if (e == cudaSuccess) e = cudaMemset(plan->d_err, 0, 4);
    if (e != cudaSuccess) return e;
    return bconv_tc_upload(plan, h);
}

// ModUp of hybrid key switching: digit j (limbs [lo, hi) of Q, alpha per digit) converts to
// every other limb of Q u P, in Q u P order; its own limbs are the skipped rows.
cudaError_t modup_plan_upload(hefx_modup_plan* mp) {
    const uint32_t L = mp->L;
    std::vector<BConvConst> h(mp->dnum);
    std::vector<uint32_t> qp(mp->q);
    qp.insert(qp.end(), mp->p.begin(), mp->p.end());
    for (uint32_t j = 0; j < mp->dnum; ++j) {
        const uint32_t lo = j * mp->alpha, hi = std::min(L, lo + mp->alpha);
        std::vector<uint32_t> dst(qp.begin(), qp.begin() + lo);
        dst.insert(dst.end(), qp.begin() + hi, qp.end());
        fill_bconv_const(mp->q.data() + lo, hi - lo, dst.data(), (uint32_t)dst.size(), h[j]);
        h[j].skip_lo = lo;
        h[j].skip_len = hi - lo;
    }
    cudaError_t e = cudaMalloc(&mp->d_const, sizeof(BConvConst) * mp->dnum);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(mp->d_const, h.data(), sizeof(BConvConst) * mp->dnum, cudaMemcpyHostToDevice);
}

void bconv_plan_free(hefx_bconv_plan* plan) {
    if (plan->d_const) cudaFree(plan->d_const);
    plan->d_const = nullptr;
    if (plan->d_err) cudaFree(plan->d_err);
    plan->d_err = nullptr;
    bconv_tc_free(plan);
}

namespace {

constexpr int kJChunk = 8;  // target limbs accumulated per pass over the source limbs
constexpr int kIGroup = 8;  // source limbs whose loads are in flight together

// kCoef coefficients per thread: each constant load serves kCoef products.
// Polynomial b's source limbs start at in + b * in_stride, its outputs at out + b * out_stride.
// MODE 1 (ModDown): the epilogue returns (x_j - conv_j) * P^-1 mod p_j, x_j at
// xq + b * in_stride + j n.  MODE 2 (exact): conv_j - v [Q]_{p_j}, v = round(sum_i b_i / q_i).
// A persistent grid (at most the resident blocks of every SM) strides over (target chunk,
// coefficient group) pairs, so each block copies the plan constants to shared memory once
// and a conversion of one polynomial to many targets still fills the GPU.
// MODE 3 (ModUp): block row y converts digit y of a ModUp plan (constants gc[y], sources the
// input rows from skip_lo, outputs at out + y * out_digit_stride with the digit's own rows
// skipped); the threads of target chunk 0 also copy the digit's own limbs into those rows.
// MODE 4 (list): block row y converts one polynomial of an independent conversion of its own
// (BcListEntry y: plan constants, source and output pointers; serving batches requests whose
// source bases differ).
enum : int { BC_FAST = 0, BC_MODDOWN = 1, BC_EXACT = 2, BC_MODUP = 3, BC_LIST = 4 };

template <int kCoef>
__host__ __device__ constexpr int log2_const() {
    return kCoef == 1 ? 0 : 1 + log2_const<kCoef / 2>();
}

// Step 1 and step 2 of one source limb i for kCoef coefficients.
template <int kCoef>
__device__ __forceinline__ void bconv_limb(const BConvConst& c, uint32_t i, uint32_t j0, const uint32_t (&x)[kCoef],
                                           uint64_t (&acc)[kCoef][kJChunk]) {
    const uint4 qc = *reinterpret_cast<const uint4*>(c.qpack[i]);  // q_i, qhat_i^-1, Shoup companion
    // kJChunk = 8 consecutive words of row i: two 16-byte shared loads
    const uint4* row = reinterpret_cast<const uint4*>(&c.qhat_p[i * kBConvMaxLimbs + j0]);
    const uint4 r0 = row[0], r1 = row[1];
    const uint32_t cst[kJChunk] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
    for (int u = 0; u < kCoef; ++u) {
        const uint32_t bi = csub(mul_shoup_lazy(x[u], qc.y, qc.z, qc.x), qc.x);  // step 1
#pragma unroll
        for (int jj = 0; jj < kJChunk; ++jj) acc[u][jj] += (uint64_t)bi * cst[jj];  // step 2
    }
}

// Exact conversion: accumulate b_i round(2^k / q_i) into a 128-bit (hi, lo) sum.
__device__ __forceinline__ void exact_limb(const BConvConst& c, uint32_t i, uint32_t x, uint64_t& lo, uint64_t& hi) {
    const uint4 qc = *reinterpret_cast<const uint4*>(c.qpack[i]);
    const uint32_t bi = csub(mul_shoup_lazy(x, qc.y, qc.z, qc.x), qc.x);
    const uint64_t plo = (uint64_t)bi * c.w[i], phi = __umul64hi((uint64_t)bi, c.w[i]);
    lo += plo;
    hi += phi + (lo < plo ? 1u : 0u);
}

// LOGN > 0 fixes the ring degree at compile time (the loads of a group then sit at constant
// offsets from one pointer); LOGN = 0 takes it from log2n.
// ModUp: 4 resident blocks per SM (its digit-copy stores spill at 48 registers; measured
// 49.8 vs 51.8 us for three 16 -> 48 digits at N = 2^16); every other mode 5.
template <int kCoef, int MODE, int LOGN>
__global__ void __launch_bounds__(256, MODE == BC_MODUP ? 4 : 5)
    bconv_cc_kernel(const BConvConst* __restrict__ gc, const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                    const uint32_t* __restrict__ xq, uint32_t log2n, uint32_t batch, size_t in_stride,
                    size_t out_stride, size_t out_digit_stride) {
    static_assert((kCoef & (kCoef - 1)) == 0, "kCoef is a power of two");
    __shared__ __align__(16) BConvConst c;
    if constexpr (MODE == BC_MODUP) gc += blockIdx.y;
    if constexpr (MODE == BC_LIST) {
        const BcListEntry e = reinterpret_cast<const BcListEntry*>(gc)[blockIdx.y];
        gc = static_cast<const BConvConst*>(e.c);
        in = e.in;
        out = e.out;
    }
    {
        // the vectors, then the L used rows of the step 2 matrix
        const uint32_t L = __ldg(&gc->L);
        const uint32_t words = (uint32_t)(offsetof(BConvConst, qhat_p) / 4) + L * kBConvMaxLimbs;
        const uint4* s4 = reinterpret_cast<const uint4*>(gc);
        uint4* d4 = reinterpret_cast<uint4*>(&c);
        for (uint32_t k = threadIdx.x; k < words / 4; k += blockDim.x) d4[k] = __ldg(s4 + k);
    }
    __syncthreads();
    // the plan constants are written once at plan creation; everything below waits for the
    // stream's preceding kernel (programmatic dependent launch)
    griddep_wait();
    if (LOGN > 0) log2n = LOGN;
    const uint32_t L = c.L, Lp = c.Lp;
    if constexpr (MODE == BC_MODUP) {
        in += (size_t)c.skip_lo << log2n;
        out += blockIdx.y * out_digit_stride;
    }
    const uint32_t lpp = log2n - log2_const<kCoef>();  // n is a multiple of kCoef
    const size_t per_poly = (size_t)1 << lpp, n = (size_t)1 << log2n;
    const size_t groups = (size_t)batch << lpp;
    const uint32_t Lfull = L - L % kIGroup;  // limbs in full groups
    // one thread per (chunk of kJChunk target limbs, group of kCoef coefficients): the group is
    // the fast index, so the lanes of a warp read consecutive coefficients
    const uint32_t nchunks = (Lp + kJChunk - 1) / kJChunk;
    // grid-stride over (chunk, group) pairs, chunk-major; the pair advances by a fixed
    // (chunk, group) step, so there is no division per task
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t first = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const uint32_t cstep = (uint32_t)(stride / groups);
    const size_t tstep = stride - (size_t)cstep * groups;
    uint32_t chunk = (uint32_t)(first / groups);
    size_t t = first - (size_t)chunk * groups;
    while (chunk < nchunks) {
        const uint32_t j0 = chunk * kJChunk;
        {
            // kCoef coefficients x, x + stride, ... of one polynomial (stride keeps warps coalesced)
            const size_t b = t >> lpp, x0 = t & (per_poly - 1);
            const uint32_t* src = in + b * in_stride + x0;
            uint32_t* dst = out + b * out_stride + x0;
            uint32_t v[kCoef];  // exact conversion: the multiple of Q to remove
            if constexpr (MODE == BC_EXACT) {
#pragma unroll
                for (int u = 0; u < kCoef; ++u) {
                    uint64_t lo = c.half_lo, hi = c.half_hi;
                    const uint32_t* p = src + u * per_poly;
                    uint32_t i0 = 0;
                    for (; i0 < Lfull; i0 += kIGroup, p += kIGroup * n) {
                        uint32_t xg[kIGroup];
#pragma unroll
                        for (int g = 0; g < kIGroup; ++g) xg[g] = __ldg(p + g * n);
#pragma unroll
                        for (int g = 0; g < kIGroup; ++g) exact_limb(c, i0 + g, xg[g], lo, hi);
                    }
                    for (; i0 < L; ++i0, p += n) exact_limb(c, i0, __ldg(p), lo, hi);
                    v[u] = (uint32_t)(hi >> c.kshift);
                }
            }
            uint64_t acc[kCoef][kJChunk];
#pragma unroll
            for (int u = 0; u < kCoef; ++u)
#pragma unroll
                for (int jj = 0; jj < kJChunk; ++jj) acc[u][jj] = 0;
            // groups of kIGroup source limbs: the group's loads are all in flight before its
            // arithmetic, so a thread waits for one DRAM round trip per group, not per limb;
            // full groups need no bounds checks
            const uint32_t* p = src;
            uint32_t i0 = 0;
            for (; i0 < Lfull; i0 += kIGroup, p += kIGroup * n) {
                uint32_t x[kIGroup][kCoef];
#pragma unroll
                for (int g = 0; g < kIGroup; ++g)
#pragma unroll
                    for (int u = 0; u < kCoef; ++u) x[g][u] = __ldg(p + g * n + u * per_poly);
#pragma unroll
                for (int g = 0; g < kIGroup; ++g) bconv_limb<kCoef>(c, i0 + g, j0, x[g], acc);
                if (MODE == BC_MODUP && j0 == 0)
#pragma unroll
                    for (int g = 0; g < kIGroup; ++g)
#pragma unroll
                        for (int u = 0; u < kCoef; ++u) dst[(size_t)(c.skip_lo + i0 + g) * n + u * per_poly] = x[g][u];
            }
            if (i0 < L) {  // the ragged last group
                uint32_t x[kIGroup][kCoef];
#pragma unroll
                for (int g = 0; g < kIGroup; ++g)
#pragma unroll
                    for (int u = 0; u < kCoef; ++u) x[g][u] = i0 + g < L ? __ldg(p + g * n + u * per_poly) : 0u;
#pragma unroll
                for (int g = 0; g < kIGroup; ++g)
                    if (i0 + g < L) bconv_limb<kCoef>(c, i0 + g, j0, x[g], acc);
                if (MODE == BC_MODUP && j0 == 0)
#pragma unroll
                    for (int g = 0; g < kIGroup; ++g)
                        if (i0 + g < L)
#pragma unroll
                            for (int u = 0; u < kCoef; ++u)
                                dst[(size_t)(c.skip_lo + i0 + g) * n + u * per_poly] = x[g][u];
            }
#pragma unroll
            for (int jj = 0; jj < kJChunk; ++jj) {
                const uint32_t j = j0 + jj;
                if (j < Lp) {
#pragma unroll
                    for (int u = 0; u < kCoef; ++u) {
                        uint32_t r = barrett64(acc[u][jj], c.p[j], c.p_mu[j]);
                        if constexpr (MODE == BC_EXACT) {
                            const uint32_t corr = barrett64((uint64_t)v[u] * c.qmod_p[j], c.p[j], c.p_mu[j]);
                            r = csub(r + c.p[j] - corr, c.p[j]);
                        }
                        if constexpr (MODE == BC_MODDOWN) {
                            const uint32_t pj = c.p[j];
                            const uint32_t xj = __ldg(xq + b * in_stride + (size_t)j * n + x0 + u * per_poly);
                            r = csub(mul_shoup_lazy(xj + pj - r, c.pinv[j], c.pinv_sh[j], pj), pj);
                        }
                        const uint32_t jr = MODE == BC_MODUP && j >= c.skip_lo ? j + c.skip_len : j;
                        dst[(size_t)jr * n + u * per_poly] = r;
                    }
                }
            }
        }
        t += tstep;  // t + tstep < 2 groups
        chunk += cstep;
        if (t >= groups) {
            t -= groups;
            ++chunk;
        }
    }
}

// Persistent grid: at most the resident blocks of every SM (occupancy cached per instance).
template <int kCoef, int MODE, int LOGN>
unsigned bconv_blocks(size_t total, uint32_t Lp) {
    static int resident[64];  // blocks per SM x SMs, per device ordinal; 0 = not yet known
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (resident[dev] == 0) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bconv_cc_kernel<kCoef, MODE, LOGN>, 256, 0) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm <= 0 || sms <= 0)
            per_sm = 1, sms = 148;
        resident[dev] = per_sm * sms;
    }
    const size_t blocks = (total / kCoef * ((Lp + kJChunk - 1) / kJChunk) + 255) / 256;
    return (unsigned)std::min(blocks, (size_t)resident[dev]);
}

}  // namespace

namespace {

// The N = 2^16 instance has the ring degree compiled in; every other degree takes the generic one.
// One coefficient per thread and 5 resident blocks per SM (48 registers) measured best on
// the conversions of HE-Mult (ModUp 16 -> 48 limbs, ModDown 16 -> 48 limbs of two
// polynomials); 2 coefficients per thread gained 4% on 24 -> 8 limbs but lost on ModUp.
template <int MODE>
cudaError_t launch_cc(const hefx_bconv_plan* plan, const uint32_t* in, uint32_t* out, const uint32_t* xq, size_t batch,
                      size_t in_stride, cudaStream_t stream) {
    const size_t total = ((size_t)1 << plan->log2n) * batch;
    const size_t out_stride = (size_t)plan->Lp << plan->log2n;
    const BConvConst* gc = static_cast<const BConvConst*>(plan->d_const);
    if (plan->log2n == 16)
        return launch_pdl(bconv_cc_kernel<1, MODE, 16>, dim3(bconv_blocks<1, MODE, 16>(total, plan->Lp)), dim3(256), 0,
                          stream, gc, in, out, xq, plan->log2n, (uint32_t)batch, in_stride, out_stride, (size_t)0);
    return launch_pdl(bconv_cc_kernel<1, MODE, 0>, dim3(bconv_blocks<1, MODE, 0>(total, plan->Lp)), dim3(256), 0,
                      stream, gc, in, out, xq, plan->log2n, (uint32_t)batch, in_stride, out_stride, (size_t)0);
}

}  // namespace

cudaError_t launch_mod_up(const hefx_modup_plan* mp, const uint32_t* c, uint32_t* U, size_t batch,
                          cudaStream_t stream) {
    if (batch == 0) return cudaSuccess;
    const size_t n = (size_t)1 << mp->log2n;
    const uint32_t rows = mp->L + mp->K;                       // rows of one digit's output
    const uint32_t lp_max = rows - std::min(mp->alpha, mp->L);  // targets of a full digit (the most)
    const size_t in_stride = (size_t)mp->L * n, digit_stride = (size_t)rows * n;
    const size_t out_stride = digit_stride * mp->dnum;
    const size_t total = n * batch;
    // the resident blocks of the GPU shared between the digits (block row y = digit y)
    const unsigned all = mp->log2n == 16 ? bconv_blocks<1, BC_MODUP, 16>(total * mp->dnum, lp_max)
                                         : bconv_blocks<1, BC_MODUP, 0>(total * mp->dnum, lp_max);
    const dim3 grid(std::max(1u, all / mp->dnum), mp->dnum);
    const BConvConst* gc = static_cast<const BConvConst*>(mp->d_const);
    const uint32_t* none = nullptr;
    if (mp->log2n == 16)
        return launch_pdl(bconv_cc_kernel<1, BC_MODUP, 16>, grid, dim3(256), 0, stream, gc, c, U, none, mp->log2n,
                          (uint32_t)batch, in_stride, out_stride, digit_stride);
    return launch_pdl(bconv_cc_kernel<1, BC_MODUP, 0>, grid, dim3(256), 0, stream, gc, c, U, none, mp->log2n,
                      (uint32_t)batch, in_stride, out_stride, digit_stride);
}

cudaError_t launch_bconv_cc_list(const BcListEntry* d_list, uint32_t count, uint32_t log2n, uint32_t lp_max,
                                 cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    const size_t n = (size_t)1 << log2n;
    const unsigned all = log2n == 16 ? bconv_blocks<1, BC_LIST, 16>(n * count, lp_max)
                                     : bconv_blocks<1, BC_LIST, 0>(n * count, lp_max);
    const dim3 grid(std::max(1u, all / count), count);
    const BConvConst* gc = reinterpret_cast<const BConvConst*>(d_list);
    const uint32_t* none = nullptr;
    uint32_t* nout = nullptr;
    if (log2n == 16)
        return launch_pdl(bconv_cc_kernel<1, BC_LIST, 16>, grid, dim3(256), 0, stream, gc, none, nout, none, log2n,
                          1u, (size_t)0, (size_t)0, (size_t)0);
    return launch_pdl(bconv_cc_kernel<1, BC_LIST, 0>, grid, dim3(256), 0, stream, gc, none, nout, none, log2n, 1u,
                      (size_t)0, (size_t)0, (size_t)0);
}

// The plain conversion takes the TMA-fed kernel (bconv_cc_tma.cu) where it applies.
#ifndef HEFX_BC_TMA
#define HEFX_BC_TMA 1
#endif

cudaError_t launch_bconv_cc(const hefx_bconv_plan* plan, const uint32_t* in, uint32_t* out, size_t batch,
                            cudaStream_t stream) {
    if (batch == 0) return cudaSuccess;
    if (HEFX_BC_TMA) {
        const cudaError_t e = launch_bconv_cc_tma(plan, in, out, batch, plan->d_err, stream);
        if (e != cudaErrorNotSupported) return e;
    }
    return launch_cc<BC_FAST>(plan, in, out, nullptr, batch, (size_t)plan->L << plan->log2n, stream);
}

cudaError_t launch_bconv_exact(const hefx_bconv_plan* plan, const uint32_t* in, uint32_t* out, size_t batch,
                               cudaStream_t stream) {
    if (batch == 0) return cudaSuccess;
    return launch_cc<BC_EXACT>(plan, in, out, nullptr, batch, (size_t)plan->L << plan->log2n, stream);
}

cudaError_t launch_mod_down(const hefx_bconv_plan* plan, const uint32_t* x, uint32_t* out, size_t batch,
                            cudaStream_t stream) {
    // x: [batch][Lp + L][n] (target-basis limbs first, then the plan's source limbs)
    if (batch == 0) return cudaSuccess;
    const size_t n = (size_t)1 << plan->log2n;
    return launch_cc<BC_MODDOWN>(plan, x + (size_t)plan->Lp * n, out, x, batch, (size_t)(plan->L + plan->Lp) * n,
                                 stream);
}

}  // namespace hefx
