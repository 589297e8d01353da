// hefx C ABI: argument validation, parameter-set precompute and dispatch.
//
// Every entry point validates on the host, returns a status without launching anything
// on error, and otherwise enqueues its kernels on the caller's stream.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <set>

#include "bconv_common.h"
#include "hefx_internal.h"
#include "host_nt.h"

using namespace hefx;

namespace {

hefx_status fail(hefx_ctx* ctx, hefx_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->last_error = buf;
    }
    return st;
}

hefx_status cuda_fail(hefx_ctx* ctx, cudaError_t e, const char* what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? HEFX_ENOMEM : HEFX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// True when [a, a + an) and [b, b + bn) (bytes) overlap.
bool overlaps(const void* a, size_t an, const void* b, size_t bn) {
    const char *x = (const char*)a, *y = (const char*)b;
    return an && bn && x < y + bn && y < x + an;
}

hefx_status use_device(hefx_ctx* ctx) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess && cur != ctx->device) e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return HEFX_OK;
}

hefx_status check_ntt_args(hefx_ctx* ctx, const hefx_params* p, const void* ptr, const char* name) {
    if (!ctx) return HEFX_EINVAL;
    if (!p || p->ctx != ctx) return fail(ctx, HEFX_EINVAL, "params is null or belongs to another context");
    if (!ptr) return fail(ctx, HEFX_EINVAL, "%s is null", name);
    if (!aligned16(ptr)) return fail(ctx, HEFX_EINVAL, "%s is not 16-byte aligned", name);
    return HEFX_OK;
}

// The tensor path is taken only where it is built for the shape; AUTO follows the tuner's
// measured choice (set from Python after timing both paths), else the CUDA-core path.
hefx_path resolve(const hefx_params* p, hefx_path path) {
    if (path == HEFX_PATH_AUTO) {
        if (p->tuned_path == HEFX_PATH_TENSOR && tc_supported(p)) return HEFX_PATH_TENSOR;
        return HEFX_PATH_CUDACORE;
    }
    return path;
}

hefx_status ensure_tc(hefx_ctx* ctx, const hefx_params* pc) {
    hefx_params* p = const_cast<hefx_params*>(pc);
    if (!tc_supported(p))
        return fail(ctx, HEFX_EUNSUPPORTED, "tensor path not available for N = 2^%u with these moduli", p->log2n);
    std::lock_guard<std::mutex> g(p->tc_mu);
    if (!p->tc && tc_narrow(p)) {  // the single-pass form's tables (no-allocation product)
        cudaError_t e = tc_prepare(p);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-path tables");
    }
    if (!p->tc2) {
        cudaError_t e = tc2_prepare(p);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-path tables (pipelined)");
    }
    return HEFX_OK;
}

RowDesc row_desc(const hefx_params* p, uint32_t l, const uint32_t* in, const uint32_t* had, uint32_t* out) {
    RowDesc r;
    memset(&r, 0, sizeof r);
    r.in = in;
    r.had = had;
    r.out = out;
    r.lc = p->d_lc + l;
    r.twf = p->d_tw_fwd + (size_t)l * p->n;
    r.twi = p->d_tw_inv + (size_t)l * p->n;
    r.limb = l;
    return r;
}

// Fused batch plan: rows grouped by (ring degree, second-half kind), cut into cluster tasks of
// 2^16 elements (ntt_cc_batch_rows_per_task rows), largest ring degree first.  The last task
// of a split ring degree (2^14 .. 2^16, whose CTAs exchange data inside the cluster) is filled
// with scratch rows so that every CTA of the cluster runs the same barriers.
typedef std::vector<std::pair<RowDesc, RowDesc>> RowPairs;  // (first half, second half) per row

hefx_status batch_plan_fused(hefx_ctx* ctx, const std::vector<const hefx_params*>& order,
                             const std::vector<RowPairs>& pfhi, const std::vector<RowPairs>& psq, hefx_batch_plan** out) {
    hefx_batch_plan* plan = new hefx_batch_plan();
    plan->ctx = ctx;
    plan->fused = true;
    plan->err = order[0]->d_err_cc;
    std::vector<size_t> idx(order.size());
    for (size_t g = 0; g < idx.size(); ++g) idx[g] = g;
    std::sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return order[x]->log2n > order[y]->log2n; });
    // scratch for fill rows: a, b, c of the largest ring degree
    uint32_t nmax = 0;
    for (const hefx_params* pr : order) nmax = std::max(nmax, pr->n);
    cudaError_t e = cudaMalloc(&plan->d_pad, 3ull * nmax * 4);
    if (e == cudaSuccess) e = cudaMemset(plan->d_pad, 0, 3ull * nmax * 4);
    if (e != cudaSuccess) {
        hefx_batch_plan_destroy(plan);
        return cuda_fail(ctx, e, "batch plan scratch");
    }
    std::vector<RowDesc> first, second;
    std::vector<BatchTask> tasks;
    for (size_t g : idx) {
        const hefx_params* pr = order[g];
        const uint32_t per = ntt_cc_batch_rows_per_task(pr->log2n);
        const bool split = pr->log2n >= 14;
        for (int kind = 0; kind < 2; ++kind) {
            const RowPairs& pairs = kind == 0 ? pfhi[g] : psq[g];
            size_t nrows = pairs.size();
            if (nrows == 0) continue;
            std::vector<RowDesc> one, t2;
            for (const auto& pr2 : pairs) {
                one.push_back(pr2.first);
                t2.push_back(pr2.second);
            }
            if (split && nrows % per) {
                uint32_t* pa = plan->d_pad;
                uint32_t* pb = plan->d_pad + nmax;
                uint32_t* pc = plan->d_pad + 2ull * nmax;
                while (nrows % per) {
                    one.push_back(row_desc(pr, 0, pa, nullptr, pc));
                    t2.push_back(kind == 0 ? row_desc(pr, 0, pb, pc, pc) : row_desc(pr, 0, pc, pc, pc));
                    ++nrows;
                }
            }
            for (size_t r = 0; r < nrows; r += per) {
                BatchTask t;
                t.logn = pr->log2n;
                t.mode = kind == 0 ? MODE_FWD_HAD_INV : MODE_HAD_INV;
                t.row0 = (uint32_t)(first.size() + r);
                t.nrows = (uint32_t)std::min<size_t>(per, nrows - r);
                tasks.push_back(t);
            }
            first.insert(first.end(), one.begin(), one.end());
            second.insert(second.end(), t2.begin(), t2.end());
        }
    }
    plan->off2 = (uint32_t)first.size();
    plan->ntasks = (uint32_t)tasks.size();
    plan->total_rows = first.size();
    std::vector<RowDesc> all = first;
    all.insert(all.end(), second.begin(), second.end());
    e = cudaMalloc(&plan->d_rows, all.size() * sizeof(RowDesc));
    if (e == cudaSuccess) e = cudaMemcpy(plan->d_rows, all.data(), all.size() * sizeof(RowDesc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&plan->d_tasks, tasks.size() * sizeof(BatchTask));
    if (e == cudaSuccess)
        e = cudaMemcpy(plan->d_tasks, tasks.data(), tasks.size() * sizeof(BatchTask), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        hefx_batch_plan_destroy(plan);
        return cuda_fail(ctx, e, "batch plan upload");
    }
    *out = plan;
    return HEFX_OK;
}

}  // namespace

// Native form of the serving request (HE-Mult front half; see hefx_mult_front in hefx.h):
// the parameter sets, conversion plan and key buffers belong to the caller.
struct hefx_mult_plan {
    hefx_ctx* ctx = nullptr;
    const hefx_params* pq = nullptr;
    const hefx_params* pp = nullptr;
    const hefx_bconv_plan* bc = nullptr;
    const uint32_t* kq[2] = {nullptr, nullptr};
    const uint32_t* kp[2] = {nullptr, nullptr};
};

namespace hefx {
bool mult_plan_view(const hefx_mult_plan* plan, MultPlanView* out) {
    if (!plan) return false;
    out->ctx = plan->ctx;
    out->pq = plan->pq;
    out->pp = plan->pp;
    out->bc = plan->bc;
    for (int k = 0; k < 2; ++k) {
        out->kq[k] = plan->kq[k];
        out->kp[k] = plan->kp[k];
    }
    return true;
}
}  // namespace hefx

extern "C" {

const char* hefx_version(void) { return "hefx 0.1 (sm_103a)"; }

hefx_status hefx_create(hefx_ctx** out, int device) {
    if (!out) return HEFX_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return HEFX_ECUDA;
    hefx_ctx* c = new hefx_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    *out = c;
    return HEFX_OK;
}

void hefx_destroy(hefx_ctx* ctx) { delete ctx; }

const char* hefx_last_error(const hefx_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

hefx_status hefx_params_create(hefx_ctx* ctx, uint32_t log2n, const uint32_t* primes, uint32_t nlimbs,
                               hefx_params** out) {
    if (!ctx || !out) return HEFX_EINVAL;
    *out = nullptr;
    if (log2n < 3 || log2n > 17) return fail(ctx, HEFX_EUNSUPPORTED, "log2n = %u outside [3, 17]", log2n);
    if (!primes || nlimbs == 0 || nlimbs > 4096) return fail(ctx, HEFX_EINVAL, "need 1..4096 primes");
    const uint64_t n = 1ull << log2n;
    std::set<uint32_t> seen;
    for (uint32_t i = 0; i < nlimbs; ++i) {
        const uint32_t q = primes[i];
        if (q < 17 || q >= (1u << 30) || !is_prime(q))
            return fail(ctx, HEFX_EINVAL, "primes[%u] = %u is not a prime in [17, 2^30)", i, q);
        if ((q - 1) % (2 * n) != 0) return fail(ctx, HEFX_EINVAL, "primes[%u] = %u is not 1 mod 2N", i, q);
        if (!seen.insert(q).second) return fail(ctx, HEFX_EINVAL, "primes[%u] = %u repeats", i, q);
    }
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;

    hefx_params* p = new hefx_params();
    p->ctx = ctx;
    p->log2n = log2n;
    p->n = (uint32_t)n;
    p->nlimbs = nlimbs;
    p->primes.assign(primes, primes + nlimbs);
    for (uint32_t i = 0; i < nlimbs; ++i) p->max_prime = std::max(p->max_prime, primes[i]);
    std::vector<LimbConst> lc(nlimbs);
    std::vector<uint2> twf((size_t)nlimbs * n), twi((size_t)nlimbs * n);
    const bool two_pass = log2n == 16;
    std::vector<uint2> twf2(two_pass ? twf.size() : 0), twi2(two_pass ? twi.size() : 0);
    std::vector<uint64_t> pw(n), pwi(n);
    for (uint32_t l = 0; l < nlimbs; ++l) {
        const uint64_t q = primes[l];
        const uint64_t psi = root_2n(q, n), psi_inv = inv_mod(psi, q);
        p->psi.push_back((uint32_t)psi);
        pw[0] = pwi[0] = 1;
        for (uint64_t e = 1; e < n; ++e) {
            pw[e] = mul_mod(pw[e - 1], psi, q);
            pwi[e] = mul_mod(pwi[e - 1], psi_inv, q);
        }
        // Twiddle tables in bit-reversed order (entry k = psi^(+-brv(k))), except that the
        // stages of the smallest-stride register pass are stored group-major: the group
        // G = J 2^v + g of sub-transform J sits at stage_base + g * (N / 2^RS) + J, so the
        // lanes of a warp (consecutive J) read consecutive entries (MAT's offline
        // reordering of constants, Sec. IV-B, applied to the table layout).
        // The two-pass transform at N = 2^16 (ntt_cc_2p.cu) reads a second copy whose
        // group-major part covers its 4-stage smallest-stride pass.
        auto fwd_pos = [&](uint64_t k, int RS) -> uint64_t {
            if (k == 0) return 0;
            int s = 63 - __builtin_clzll(k);  // stage of entry k: k in [2^s, 2^(s+1))
            if (s < (int)log2n - RS) return k;
            const int v = s - ((int)log2n - RS);
            const uint64_t G = k - (1ull << s), J = G >> v, g = G & ((1ull << v) - 1);
            return (1ull << s) + g * (n >> RS) + J;
        };
        auto inv_pos = [&](uint64_t k, int RS) -> uint64_t {
            if (k == 0) return 0;
            int hb = 63 - __builtin_clzll(k);  // entry k belongs to stage e = log2n - 1 - hb
            const int e = (int)log2n - 1 - hb;
            if (e >= RS) return k;
            const int w = RS - 1 - e;
            const uint64_t G = k - (1ull << hb), J = G >> w, g = G & ((1ull << w) - 1);
            return (1ull << hb) + g * (n >> RS) + J;
        };
        const int RS = ntt_cc_small_radix((int)log2n);
        for (uint64_t k = 0; k < n; ++k) {
            const uint32_t r = bit_reverse((uint32_t)k, (int)log2n);
            const uint2 wf = make_uint2((uint32_t)pw[r], shoup(pw[r], q));
            const uint2 wi = make_uint2((uint32_t)pwi[r], shoup(pwi[r], q));
            twf[l * n + fwd_pos(k, RS)] = wf;
            twi[l * n + inv_pos(k, RS)] = wi;
            if (two_pass) {
                twf2[l * n + fwd_pos(k, 4)] = wf;
                twi2[l * n + inv_pos(k, 4)] = wi;
            }
        }
        LimbConst& c = lc[l];
        memset(&c, 0, sizeof c);
        c.q = (uint32_t)q;
        c.qinv_neg = neg_inv_pow2_32((uint32_t)q);
        const uint64_t ninv = inv_mod(n % q, q);
        const uint64_t w1 = pwi[bit_reverse(1, (int)log2n)];  // psi^-(N/2), last Gentleman-Sande twiddle
        const uint64_t r32 = ((uint64_t)1 << 32) % q;
        const uint64_t vals[4] = {ninv, mul_mod(ninv, w1, q), mul_mod(ninv, r32, q),
                                  mul_mod(mul_mod(ninv, r32, q), w1, q)};
        c.ninv = (uint32_t)vals[0];
        c.ninv_sh = shoup(vals[0], q);
        c.ninvw = (uint32_t)vals[1];
        c.ninvw_sh = shoup(vals[1], q);
        c.ninvR = (uint32_t)vals[2];
        c.ninvR_sh = shoup(vals[2], q);
        c.ninvRw = (uint32_t)vals[3];
        c.ninvRw_sh = shoup(vals[3], q);
        c.r2 = (uint32_t)mul_mod(r32, r32, q);
        c.one_sh = shoup(1, q);
        c.q2 = (uint32_t)(2 * q);
        c.q4 = (uint32_t)(4 * q);
        c.q8 = (uint32_t)(8 * q);  // wraps for q >= 2^29: used only where q < 2^28 (lazy ranges)
        const uint64_t mu = (uint64_t)((((unsigned __int128)1) << 64) / q);
        c.bar_lo = (uint32_t)mu;
        c.bar_hi = (uint32_t)(mu >> 32);
        if (l + 1 < nlimbs) {
            const uint64_t ri = inv_mod(primes[nlimbs - 1] % q, q);
            c.rs_inv = (uint32_t)ri;
            c.rs_inv_sh = shoup(ri, q);
        }
    }
    cudaError_t e = cudaMalloc(&p->d_lc, sizeof(LimbConst) * nlimbs);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_err_cc, 4);
    if (e == cudaSuccess) e = cudaMemset(p->d_err_cc, 0, 4);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tw_fwd, sizeof(uint2) * twf.size());
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tw_inv, sizeof(uint2) * twi.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->d_lc, lc.data(), sizeof(LimbConst) * nlimbs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_tw_fwd, twf.data(), sizeof(uint2) * twf.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_tw_inv, twi.data(), sizeof(uint2) * twi.size(), cudaMemcpyHostToDevice);
    if (two_pass) {
        if (e == cudaSuccess) e = cudaMalloc(&p->d_tw2_fwd, sizeof(uint2) * twf2.size());
        if (e == cudaSuccess) e = cudaMalloc(&p->d_tw2_inv, sizeof(uint2) * twi2.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_tw2_fwd, twf2.data(), sizeof(uint2) * twf2.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_tw2_inv, twi2.data(), sizeof(uint2) * twi2.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        hefx_params_destroy(p);
        return cuda_fail(ctx, e, "parameter tables");
    }
    *out = p;
    return HEFX_OK;
}

void hefx_params_destroy(hefx_params* p) {
    if (!p) return;
    if (p->ctx) {
        int cur = -1;
        if (cudaGetDevice(&cur) == cudaSuccess && cur != p->ctx->device) cudaSetDevice(p->ctx->device);
    }
    tc_free(p);
    if (p->d_lc) cudaFree(p->d_lc);
    if (p->d_tw_fwd) cudaFree(p->d_tw_fwd);
    if (p->d_tw_inv) cudaFree(p->d_tw_inv);
    if (p->d_tw2_fwd) cudaFree(p->d_tw2_fwd);
    if (p->d_tw2_inv) cudaFree(p->d_tw2_inv);
    if (p->d_err_cc) cudaFree(p->d_err_cc);
    if (p->d_tw_fwd_mont) cudaFree(p->d_tw_fwd_mont);
    if (p->d_tw_inv_mont) cudaFree(p->d_tw_inv_mont);
    delete p;
}

static hefx_status run_ntt(hefx_ctx* ctx, const hefx_params* p, uint32_t* d, size_t batch, hefx_path path,
                           void* stream, NttMode mode) {
    hefx_status st = check_ntt_args(ctx, p, d, "d_data");
    if (st != HEFX_OK) return st;
    if ((st = use_device(ctx)) != HEFX_OK) return st;
    const hefx_path pth = resolve(p, path);
    if (pth == HEFX_PATH_TENSOR && p->red_ntt != HEFX_RED_SHOUP)
        return fail(ctx, HEFX_EUNSUPPORTED, "the tensor path has no NTT reduction choice");
    if (pth == HEFX_PATH_TENSOR && (st = ensure_tc(ctx, p)) != HEFX_OK) return st;
    if (batch == 0) return HEFX_OK;
    cudaError_t e;
    if (pth == HEFX_PATH_TENSOR) {
        hefx_params* pm = const_cast<hefx_params*>(p);
        e = mode == MODE_FWD ? tc2_forward(pm, d, d, 0, nullptr, batch, (cudaStream_t)stream)
                             : tc2_inverse(pm, d, d, batch, (cudaStream_t)stream);
    } else if (pth == HEFX_PATH_CUDACORE && p->red_ntt != HEFX_RED_SHOUP) {
        e = launch_ntt_cc_red(p, mode, d, batch * p->nlimbs, (cudaStream_t)stream);
        if (e == cudaErrorNotSupported)
            return fail(ctx, HEFX_EUNSUPPORTED, "non-default NTT reduction is built for N = 2^16 only");
    } else if (pth == HEFX_PATH_CUDACORE) {
        e = launch_ntt_cc(p, mode, d, nullptr, d, batch * p->nlimbs, (cudaStream_t)stream);
    } else {
        return fail(ctx, HEFX_EINVAL, "unknown path %d", (int)path);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, mode == MODE_FWD ? "hefx_ntt_fwd launch" : "hefx_ntt_inv launch");
    return HEFX_OK;
}

hefx_status hefx_ntt_fwd(hefx_ctx* ctx, const hefx_params* p, uint32_t* d, size_t batch, hefx_path path,
                         void* stream) {
    return run_ntt(ctx, p, d, batch, path, stream, MODE_FWD);
}

hefx_status hefx_ntt_inv(hefx_ctx* ctx, const hefx_params* p, uint32_t* d, size_t batch, hefx_path path,
                         void* stream) {
    return run_ntt(ctx, p, d, batch, path, stream, MODE_INV);
}

hefx_status hefx_poly_mul(hefx_ctx* ctx, const hefx_params* p, const uint32_t* a, const uint32_t* b, uint32_t* c,
                          size_t batch, hefx_path path, void* stream) {
    hefx_status st;
    if ((st = check_ntt_args(ctx, p, a, "d_a")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, b, "d_b")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, c, "d_c")) != HEFX_OK) return st;
    if ((st = use_device(ctx)) != HEFX_OK) return st;
    const hefx_path pth = resolve(p, path);
    if (pth != HEFX_PATH_CUDACORE && pth != HEFX_PATH_TENSOR) return fail(ctx, HEFX_EINVAL, "unknown path");
    if (p->red_ntt != HEFX_RED_SHOUP)
        return fail(ctx, HEFX_EUNSUPPORTED, "hefx_poly_mul uses the default (Shoup) NTT reduction only");
    if (pth == HEFX_PATH_TENSOR && (st = ensure_tc(ctx, p)) != HEFX_OK) return st;
    if (batch == 0) return HEFX_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t rows = batch * p->nlimbs;
    if (pth == HEFX_PATH_TENSOR) {
        cudaError_t e = tc2_polymul(const_cast<hefx_params*>(p), a, b, c, batch, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_poly_mul (tensor path)");
        return HEFX_OK;
    }
    auto launch = [&](NttMode m, const uint32_t* in, const uint32_t* had, uint32_t* out) {
        return launch_ntt_cc(p, m, in, had, out, rows, s);
    };
    cudaError_t e;
    if (a == b) {
        // c = INTT(NTT(a) o NTT(a))
        e = launch(MODE_FWD, a, nullptr, c);
        if (e == cudaSuccess) e = launch(MODE_HAD_INV, c, c, c);
    } else {
        if (c == b) std::swap(a, b);  // the product commutes; keep b intact while c is written
        e = launch(MODE_FWD, a, nullptr, c);                    // c = NTT(a)
        if (e == cudaSuccess) e = launch(MODE_FWD_HAD_INV, b, c, c);  // c = INTT(NTT(b) o c)
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_poly_mul launch");
    return HEFX_OK;
}

hefx_status hefx_bconv_plan_create(hefx_ctx* ctx, uint32_t log2n, const uint32_t* src, uint32_t L,
                                   const uint32_t* dst, uint32_t Lp, hefx_bconv_plan** out) {
    if (!ctx || !out) return HEFX_EINVAL;
    *out = nullptr;
    if (log2n > 24) return fail(ctx, HEFX_EUNSUPPORTED, "log2n = %u outside [0, 24]", log2n);
    if (!src || !dst || L == 0 || Lp == 0 || L > (uint32_t)kBConvMaxLimbs || Lp > (uint32_t)kBConvMaxLimbs)
        return fail(ctx, HEFX_EINVAL, "need 1..%d source and target primes", kBConvMaxLimbs);
    std::set<uint32_t> seen;
    for (uint32_t i = 0; i < L + Lp; ++i) {
        const uint32_t q = i < L ? src[i] : dst[i - L];
        if (q < 3 || q >= (1u << 30) || !is_prime(q))
            return fail(ctx, HEFX_EINVAL, "modulus %u is not a prime in [3, 2^30)", q);
        if (!seen.insert(q).second) return fail(ctx, HEFX_EINVAL, "modulus %u repeats", q);
    }
    {  // the CUDA-core kernel accumulates L products b_i [qhat_i]_{p_j} < q_i p_j in 64 bits
        uint64_t mq = 0, mp = 0;
        for (uint32_t i = 0; i < L; ++i) mq = std::max<uint64_t>(mq, src[i]);
        for (uint32_t j = 0; j < Lp; ++j) mp = std::max<uint64_t>(mp, dst[j]);
        if ((unsigned __int128)L * (mq - 1) * (mp - 1) >= ((unsigned __int128)1 << 64))
            return fail(ctx, HEFX_EUNSUPPORTED, "L * max(q) * max(p) reaches 2^64 (64-bit accumulation)");
    }
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    hefx_bconv_plan* p = new hefx_bconv_plan();
    p->ctx = ctx;
    p->log2n = log2n;
    p->L = L;
    p->Lp = Lp;
    p->src.assign(src, src + L);
    p->dst.assign(dst, dst + Lp);
    cudaError_t e = bconv_plan_upload(p);
    if (e != cudaSuccess) {
        hefx_bconv_plan_destroy(p);
        return cuda_fail(ctx, e, "basis-conversion constants");
    }
    *out = p;
    return HEFX_OK;
}

void hefx_bconv_plan_destroy(hefx_bconv_plan* p) {
    if (!p) return;
    bconv_plan_free(p);
    delete p;
}

hefx_status hefx_modup_plan_create(hefx_ctx* ctx, uint32_t log2n, const uint32_t* q, uint32_t L, const uint32_t* p,
                                   uint32_t K, uint32_t alpha, hefx_modup_plan** out) {
    if (!ctx || !out) return HEFX_EINVAL;
    *out = nullptr;
    if (log2n > 24) return fail(ctx, HEFX_EUNSUPPORTED, "log2n = %u outside [0, 24]", log2n);
    if (!q || !p || L == 0 || K == 0 || L + K > (uint32_t)kBConvMaxLimbs)
        return fail(ctx, HEFX_EINVAL, "need L >= 1, K >= 1 and L + K <= %d primes", kBConvMaxLimbs);
    if (alpha == 0 || alpha > L) return fail(ctx, HEFX_EINVAL, "alpha = %u outside [1, L]", alpha);
    std::set<uint32_t> seen;
    uint64_t mq = 0, mqp = 0;
    for (uint32_t i = 0; i < L + K; ++i) {
        const uint32_t v = i < L ? q[i] : p[i - L];
        if (v < 3 || v >= (1u << 30) || !is_prime(v))
            return fail(ctx, HEFX_EINVAL, "modulus %u is not a prime in [3, 2^30)", v);
        if (!seen.insert(v).second) return fail(ctx, HEFX_EINVAL, "modulus %u repeats", v);
        if (i < L) mq = std::max<uint64_t>(mq, v);
        mqp = std::max<uint64_t>(mqp, v);
    }
    // each digit's conversion accumulates alpha products b_i [qhat_i]_{t} < q_i t in 64 bits
    if ((unsigned __int128)alpha * (mq - 1) * (mqp - 1) >= ((unsigned __int128)1 << 64))
        return fail(ctx, HEFX_EUNSUPPORTED, "alpha * max(q) * max(q, p) reaches 2^64 (64-bit accumulation)");
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    hefx_modup_plan* mp = new hefx_modup_plan();
    mp->ctx = ctx;
    mp->log2n = log2n;
    mp->L = L;
    mp->K = K;
    mp->alpha = alpha;
    mp->dnum = (L + alpha - 1) / alpha;
    mp->q.assign(q, q + L);
    mp->p.assign(p, p + K);
    cudaError_t e = modup_plan_upload(mp);
    if (e != cudaSuccess) {
        hefx_modup_plan_destroy(mp);
        return cuda_fail(ctx, e, "ModUp constants");
    }
    *out = mp;
    return HEFX_OK;
}

void hefx_modup_plan_destroy(hefx_modup_plan* mp) {
    if (!mp) return;
    if (mp->d_const) cudaFree(mp->d_const);
    delete mp;
}

uint32_t hefx_modup_plan_dnum(const hefx_modup_plan* mp) { return mp ? mp->dnum : 0; }

hefx_status hefx_mod_up(hefx_ctx* ctx, const hefx_modup_plan* plan, const uint32_t* c, uint32_t* U, size_t batch,
                        void* stream) {
    if (!ctx) return HEFX_EINVAL;
    if (!plan || plan->ctx != ctx) return fail(ctx, HEFX_EINVAL, "plan is null or belongs to another context");
    if (!c || !U) return fail(ctx, HEFX_EINVAL, "null buffer");
    if (!aligned16(c) || !aligned16(U)) return fail(ctx, HEFX_EINVAL, "buffers must be 16-byte aligned");
    const size_t row = ((size_t)1 << plan->log2n) * 4;
    if (overlaps(U, batch * plan->dnum * (plan->L + plan->K) * row, c, batch * plan->L * row))
        return fail(ctx, HEFX_EINVAL, "d_U overlaps d_c");
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    if (batch == 0) return HEFX_OK;
    cudaError_t e = launch_mod_up(plan, c, U, batch, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_mod_up launch");
    return HEFX_OK;
}

hefx_status hefx_basis_convert(hefx_ctx* ctx, const hefx_bconv_plan* plan, const uint32_t* in, uint32_t* out,
                               size_t batch, hefx_path path, void* stream) {
    if (!ctx) return HEFX_EINVAL;
    if (!plan || plan->ctx != ctx) return fail(ctx, HEFX_EINVAL, "plan is null or belongs to another context");
    if (!in || !out) return fail(ctx, HEFX_EINVAL, "null buffer");
    if (!aligned16(in) || !aligned16(out)) return fail(ctx, HEFX_EINVAL, "buffers must be 16-byte aligned");
    const size_t n = (size_t)1 << plan->log2n;
    const char *ib = (const char*)in, *ob = (const char*)out;
    if (ib < ob + batch * plan->Lp * n * 4 && ob < ib + batch * plan->L * n * 4)
        return fail(ctx, HEFX_EINVAL, "d_out overlaps d_in");
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    if (path == HEFX_PATH_AUTO) path = bconv_prefer_tc(plan, batch) ? HEFX_PATH_TENSOR : HEFX_PATH_CUDACORE;
    if (path == HEFX_PATH_TENSOR && !bconv_tc_available(plan))
        return fail(ctx, HEFX_EUNSUPPORTED, "tensor basis conversion not available for this plan");
    if (batch == 0) return HEFX_OK;
    cudaError_t e;
    if (path == HEFX_PATH_TENSOR)
        e = launch_bconv_tc(plan, in, out, batch, (cudaStream_t)stream);
    else if (path == HEFX_PATH_CUDACORE)
        e = launch_bconv_cc(plan, in, out, batch, (cudaStream_t)stream);
    else
        return fail(ctx, HEFX_EINVAL, "unknown path %d", (int)path);
    if (e == cudaErrorNotSupported)
        return fail(ctx, HEFX_EUNSUPPORTED, "tensor basis conversion not available for this plan");
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_basis_convert launch");
    return HEFX_OK;
}

hefx_status hefx_bconv_check(hefx_ctx* ctx, const hefx_bconv_plan* plan, void* stream) {
    if (!ctx) return HEFX_EINVAL;
    if (!plan || plan->ctx != ctx) return fail(ctx, HEFX_EINVAL, "plan is null or belongs to another context");
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    uint32_t code = 0;
    cudaError_t e = cudaSuccess;
    if (plan->d_err) {
        e = cudaMemcpyAsync(&code, plan->d_err, 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e == cudaSuccess && code) e = cudaMemsetAsync(plan->d_err, 0, 4, (cudaStream_t)stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_bconv_check");
    if (code) return fail(ctx, HEFX_ETIMEOUT, "a bounded device wait of a basis conversion expired (code %u); results are invalid", code);
    return HEFX_OK;
}

hefx_status hefx_basis_convert_exact(hefx_ctx* ctx, const hefx_bconv_plan* plan, const uint32_t* in, uint32_t* out,
                                     size_t batch, void* stream) {
    if (!ctx) return HEFX_EINVAL;
    if (!plan || plan->ctx != ctx) return fail(ctx, HEFX_EINVAL, "plan is null or belongs to another context");
    if (!in || !out) return fail(ctx, HEFX_EINVAL, "null buffer");
    if (!aligned16(in) || !aligned16(out)) return fail(ctx, HEFX_EINVAL, "buffers must be 16-byte aligned");
    const size_t row = ((size_t)1 << plan->log2n) * 4;
    if (overlaps(out, batch * plan->Lp * row, in, batch * plan->L * row))
        return fail(ctx, HEFX_EINVAL, "d_out overlaps d_in");
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    if (batch == 0) return HEFX_OK;
    cudaError_t e = launch_bconv_exact(plan, in, out, batch, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_basis_convert_exact launch");
    return HEFX_OK;
}

hefx_status hefx_vec_mod_mul(hefx_ctx* ctx, const hefx_params* p, const uint32_t* x, const uint32_t* y, uint32_t* z,
                             size_t batch, void* stream) {
    hefx_status st;
    if ((st = check_ntt_args(ctx, p, x, "d_x")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, y, "d_y")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, z, "d_z")) != HEFX_OK) return st;
    if (batch == 0) return HEFX_OK;
    if ((st = use_device(ctx)) != HEFX_OK) return st;
    cudaError_t e = launch_vec_mod_mul(p, x, y, z, batch * p->nlimbs, (cudaStream_t)stream);  // p->red_vec
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_vec_mod_mul launch");
    return HEFX_OK;
}

hefx_status hefx_vec_mod_add(hefx_ctx* ctx, const hefx_params* p, const uint32_t* x, const uint32_t* y, uint32_t* z,
                             size_t batch, void* stream) {
    hefx_status st;
    if ((st = check_ntt_args(ctx, p, x, "d_x")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, y, "d_y")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, z, "d_z")) != HEFX_OK) return st;
    if (batch == 0) return HEFX_OK;
    if ((st = use_device(ctx)) != HEFX_OK) return st;
    cudaError_t e = launch_vec_mod_add(p, x, y, z, batch * p->nlimbs, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_vec_mod_add launch");
    return HEFX_OK;
}

hefx_status hefx_key_inner_product(hefx_ctx* ctx, const hefx_params* p, const uint32_t* digits, const uint32_t* evk,
                                   uint32_t* out, uint32_t dnum, size_t batch, void* stream) {
    hefx_status st;
    if ((st = check_ntt_args(ctx, p, digits, "d_digits")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, evk, "d_evk")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, out, "d_out")) != HEFX_OK) return st;
    if (dnum == 0 || dnum > 64) return fail(ctx, HEFX_EINVAL, "dnum = %u outside [1, 64]", dnum);
    const size_t poly = (size_t)p->nlimbs * p->n * 4;
    if (overlaps(out, batch * 2 * poly, digits, batch * dnum * poly) || overlaps(out, batch * 2 * poly, evk, dnum * 2 * poly))
        return fail(ctx, HEFX_EINVAL, "d_out overlaps an input");
    if (batch == 0) return HEFX_OK;
    if ((st = use_device(ctx)) != HEFX_OK) return st;
    cudaError_t e = launch_key_inner_product(p, digits, evk, out, dnum, batch, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_key_inner_product launch");
    return HEFX_OK;
}

hefx_status hefx_rescale(hefx_ctx* ctx, const hefx_params* p, const uint32_t* x, uint32_t* out, size_t batch,
                         void* stream) {
    hefx_status st;
    if ((st = check_ntt_args(ctx, p, x, "d_x")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, out, "d_out")) != HEFX_OK) return st;
    if (p->nlimbs < 2) return fail(ctx, HEFX_EINVAL, "rescale needs at least 2 limbs");
    const size_t row = (size_t)p->n * 4;
    if (!(batch == 1 && (const void*)out == (const void*)x) &&
        overlaps(out, batch * (p->nlimbs - 1) * row, x, batch * p->nlimbs * row))
        return fail(ctx, HEFX_EINVAL, "d_out overlaps d_x (in place only with batch == 1)");
    if (batch == 0) return HEFX_OK;
    if ((st = use_device(ctx)) != HEFX_OK) return st;
    cudaError_t e = launch_rescale(p, x, out, batch, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_rescale launch");
    return HEFX_OK;
}

hefx_status hefx_rescale_ntt(hefx_ctx* ctx, const hefx_params* p, const uint32_t* x, uint32_t* out, size_t batch,
                             void* stream) {
    hefx_status st;
    if ((st = check_ntt_args(ctx, p, x, "d_x")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, out, "d_out")) != HEFX_OK) return st;
    if (p->nlimbs < 2) return fail(ctx, HEFX_EINVAL, "rescale needs at least 2 limbs");
    if (p->red_ntt != HEFX_RED_SHOUP)
        return fail(ctx, HEFX_EUNSUPPORTED, "hefx_rescale_ntt uses the default (Shoup) NTT reduction only");
    const size_t row = (size_t)p->n * 4;
    if (overlaps(out, batch * (p->nlimbs - 1) * row, x, batch * p->nlimbs * row))
        return fail(ctx, HEFX_EINVAL, "d_out overlaps d_x");
    if (batch == 0) return HEFX_OK;
    if ((st = use_device(ctx)) != HEFX_OK) return st;
    cudaError_t e = launch_ntt_cc_rescale(p, x, out, batch, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_rescale_ntt launch");
    return HEFX_OK;
}

hefx_status hefx_mod_down(hefx_ctx* ctx, const hefx_bconv_plan* plan, const uint32_t* x, uint32_t* out, size_t batch,
                          void* stream) {
    if (!ctx) return HEFX_EINVAL;
    if (!plan || plan->ctx != ctx) return fail(ctx, HEFX_EINVAL, "plan is null or belongs to another context");
    if (!x || !out) return fail(ctx, HEFX_EINVAL, "null buffer");
    if (!aligned16(x) || !aligned16(out)) return fail(ctx, HEFX_EINVAL, "buffers must be 16-byte aligned");
    const size_t row = ((size_t)1 << plan->log2n) * 4;
    if (overlaps(out, batch * plan->Lp * row, x, batch * (plan->L + plan->Lp) * row))
        return fail(ctx, HEFX_EINVAL, "d_out overlaps d_x");
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    if (batch == 0) return HEFX_OK;
    cudaError_t e = launch_mod_down(plan, x, out, batch, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_mod_down launch");
    return HEFX_OK;
}

hefx_status hefx_tensor_product(hefx_ctx* ctx, const hefx_params* p, const uint32_t* a0, const uint32_t* a1,
                                const uint32_t* b0, const uint32_t* b1, uint32_t* d0, uint32_t* d1, uint32_t* d2,
                                size_t batch, void* stream) {
    const void* ptrs[7] = {a0, a1, b0, b1, d0, d1, d2};
    const char* names[7] = {"d_a0", "d_a1", "d_b0", "d_b1", "d_d0", "d_d1", "d_d2"};
    for (int i = 0; i < 7; ++i) {
        if (i == 6 && !d2) break;  // d2 not wanted
        hefx_status st = check_ntt_args(ctx, p, ptrs[i], names[i]);
        if (st != HEFX_OK) return st;
    }
    if (batch == 0) return HEFX_OK;
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    cudaError_t e = launch_tensor_product(p, a0, a1, b0, b1, d0, d1, d2, batch * p->nlimbs, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_tensor_product launch");
    return HEFX_OK;
}

hefx_status hefx_ntt_inv_hadamard(hefx_ctx* ctx, const hefx_params* p, const uint32_t* x, const uint32_t* y,
                                  uint32_t* out, size_t batch, void* stream) {
    hefx_status st;
    if ((st = check_ntt_args(ctx, p, x, "d_x")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, y, "d_y")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, out, "d_out")) != HEFX_OK) return st;
    if (p->red_ntt != HEFX_RED_SHOUP)
        return fail(ctx, HEFX_EUNSUPPORTED, "hefx_ntt_inv_hadamard uses the default (Shoup) NTT reduction only");
    const size_t bytes = batch * p->nlimbs * (size_t)p->n * 4;
    if (overlaps(out, bytes, x, bytes) || overlaps(out, bytes, y, bytes))
        return fail(ctx, HEFX_EINVAL, "d_out overlaps an input");
    if (batch == 0) return HEFX_OK;
    if ((st = use_device(ctx)) != HEFX_OK) return st;
    cudaError_t e = launch_ntt_cc(p, MODE_HAD_INV, x, y, out, batch * p->nlimbs, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_ntt_inv_hadamard launch");
    return HEFX_OK;
}

hefx_status hefx_batch_plan_create(hefx_ctx* ctx, const hefx_job* jobs, size_t njobs, hefx_path path,
                                   hefx_batch_plan** out) {
    if (!ctx || !out) return HEFX_EINVAL;
    *out = nullptr;
    if (njobs && !jobs) return fail(ctx, HEFX_EINVAL, "jobs is null");
    if (path == HEFX_PATH_TENSOR)
        return fail(ctx, HEFX_EUNSUPPORTED, "batched jobs run on the CUDA-core row-list kernels");
    if (path != HEFX_PATH_AUTO && path != HEFX_PATH_CUDACORE) return fail(ctx, HEFX_EINVAL, "unknown path");
    // group rows by (parameter set, launch kind): NTT(a) -> c; INTT(NTT(b) o c); INTT(c o c)
    std::vector<const hefx_params*> order;
    std::vector<std::vector<RowDesc>> fwd, fhi, sq;
    std::vector<RowPairs> pfhi, psq;
    for (size_t j = 0; j < njobs; ++j) {
        const hefx_job& jb = jobs[j];
        if (!jb.params || jb.params->ctx != ctx)
            return fail(ctx, HEFX_EINVAL, "job %zu: params null or of another context", j);
        if (jb.nlimbs == 0 || jb.nlimbs > jb.params->nlimbs)
            return fail(ctx, HEFX_EINVAL, "job %zu: nlimbs %u outside [1, %u]", j, jb.nlimbs, jb.params->nlimbs);
        if (!jb.d_a || !jb.d_b || !jb.d_c || !aligned16(jb.d_a) || !aligned16(jb.d_b) || !aligned16(jb.d_c))
            return fail(ctx, HEFX_EINVAL, "job %zu: null or misaligned buffer", j);
        size_t g = 0;
        while (g < order.size() && order[g] != jb.params) ++g;
        if (g == order.size()) {
            order.push_back(jb.params);
            fwd.emplace_back();
            fhi.emplace_back();
            sq.emplace_back();
            pfhi.emplace_back();
            psq.emplace_back();
        }
        const size_t n = jb.params->n;
        const uint32_t *a = jb.d_a, *b = jb.d_b;
        if (a != b && jb.d_c == b) std::swap(a, b);  // keep b intact while c is written
        for (uint32_t l = 0; l < jb.nlimbs; ++l) {
            const RowDesc r1 = row_desc(jb.params, l, a + l * n, nullptr, jb.d_c + l * n);
            fwd[g].push_back(r1);
            if (a == b) {
                const RowDesc r2 = row_desc(jb.params, l, jb.d_c + l * n, jb.d_c + l * n, jb.d_c + l * n);
                sq[g].push_back(r2);
                psq[g].push_back({r1, r2});
            } else {
                const RowDesc r2 = row_desc(jb.params, l, b + l * n, jb.d_c + l * n, jb.d_c + l * n);
                fhi[g].push_back(r2);
                pfhi[g].push_back({r1, r2});
            }
        }
    }
    // fused form when every job's ring degree and moduli suit the one-launch kernel
    bool fused = !order.empty();
    for (const hefx_params* pr : order)
        fused = fused && ntt_cc_batch_supported(pr->log2n, pr->max_prime < (1u << 28));
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    if (fused) return batch_plan_fused(ctx, order, pfhi, psq, out);
    hefx_batch_plan* plan = new hefx_batch_plan();
    plan->ctx = ctx;
    std::vector<RowDesc> all;
    auto add = [&](const hefx_params* pr, NttMode m, const std::vector<RowDesc>& rows) {
        if (rows.empty()) return;
        plan->launches.push_back({pr, (NttModeTag)m, all.size(), rows.size()});
        all.insert(all.end(), rows.begin(), rows.end());
    };
    for (size_t g = 0; g < order.size(); ++g) add(order[g], MODE_FWD, fwd[g]);
    for (size_t g = 0; g < order.size(); ++g) {
        add(order[g], MODE_FWD_HAD_INV, fhi[g]);
        add(order[g], MODE_HAD_INV, sq[g]);
    }
    plan->total_rows = all.size();
    for (const auto& l : plan->launches) {
        cudaError_t e = prepare_ntt_cc(l.params, (NttMode)l.mode);
        if (e != cudaSuccess) {
            hefx_batch_plan_destroy(plan);
            return cuda_fail(ctx, e, "batch plan kernel attributes");
        }
    }
    if (!all.empty()) {
        cudaError_t e = cudaMalloc(&plan->d_rows, all.size() * sizeof(RowDesc));
        if (e == cudaSuccess)
            e = cudaMemcpy(plan->d_rows, all.data(), all.size() * sizeof(RowDesc), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            hefx_batch_plan_destroy(plan);
            return cuda_fail(ctx, e, "batch plan upload");
        }
    }
    *out = plan;
    return HEFX_OK;
}

void hefx_batch_plan_destroy(hefx_batch_plan* plan) {
    if (!plan) return;
    if (plan->d_tasks) cudaFree(plan->d_tasks);
    if (plan->d_pad) cudaFree(plan->d_pad);
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->d_rows) cudaFree(plan->d_rows);
    delete plan;
}

uint32_t hefx_batch_plan_launches(const hefx_batch_plan* plan) {
    if (!plan) return 0;
    if (plan->fused) return plan->ntasks ? 1u : 0u;
    return (uint32_t)plan->launches.size();
}

static cudaError_t batch_launch_all(hefx_batch_plan* plan, cudaStream_t s) {
    const RowDesc* rows = static_cast<const RowDesc*>(plan->d_rows);
    if (plan->fused)
        return launch_ntt_cc_batch(rows, static_cast<const BatchTask*>(plan->d_tasks), plan->ntasks, plan->off2,
                                   plan->err, s);
    for (const auto& l : plan->launches) {
        cudaError_t e = launch_ntt_cc_rows(l.params, (NttMode)l.mode, rows + l.offset, l.nrows, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

hefx_status hefx_batch_polymul(hefx_ctx* ctx, hefx_batch_plan* plan, void* stream) {
    if (!ctx) return HEFX_EINVAL;
    if (!plan || plan->ctx != ctx) return fail(ctx, HEFX_EINVAL, "plan is null or belongs to another context");
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->launches.empty() && !(plan->fused && plan->ntasks)) return HEFX_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = s ? cudaStreamIsCapturing(s, &cap) : cudaSuccess;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamIsCapturing");
    if (!s || cap != cudaStreamCaptureStatusNone) {  // legacy stream or caller's own capture
        e = batch_launch_all(plan, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_batch_polymul launch");
        return HEFX_OK;
    }
    if (!plan->exec) {
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = batch_launch_all(plan, s);
            e = cudaStreamEndCapture(s, &plan->graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
        if (e != cudaSuccess) {
            if (plan->graph) cudaGraphDestroy(plan->graph);
            plan->graph = nullptr;
            plan->exec = nullptr;
            return cuda_fail(ctx, e, "hefx_batch_polymul graph capture");
        }
        plan->graph_stream = s;
    }
    e = cudaGraphLaunch(plan->exec, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_batch_polymul graph launch");
    return HEFX_OK;
}

hefx_status hefx_poly_mul_noalloc(hefx_ctx* ctx, const hefx_params* p, const uint32_t* a, const uint32_t* b,
                                  uint32_t* c, size_t batch, void* stream) {
    hefx_status st;
    if ((st = check_ntt_args(ctx, p, a, "d_a")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, b, "d_b")) != HEFX_OK) return st;
    if ((st = check_ntt_args(ctx, p, c, "d_c")) != HEFX_OK) return st;
    if ((st = use_device(ctx)) != HEFX_OK) return st;
    if (!tc_narrow(p))
        return fail(ctx, HEFX_EUNSUPPORTED,
                    "hefx_poly_mul_noalloc needs N = 2^14 .. 2^16 and moduli below 2^28 (N = 2^%u here)", p->log2n);
    if (p->red_ntt != HEFX_RED_SHOUP)
        return fail(ctx, HEFX_EUNSUPPORTED, "hefx_poly_mul_noalloc uses the default (Shoup) NTT reduction only");
    {
        // the tables are built under tc_mu by the first tensor-path call (ensure_tc); once
        // built they stay until hefx_params_destroy, so reading the pointer under the lock is
        // enough
        std::lock_guard<std::mutex> g(const_cast<hefx_params*>(p)->tc_mu);
        if (!p->tc)
            return fail(ctx, HEFX_EUNSUPPORTED,
                        "tensor tables of these params are not built yet; make one tensor-path call "
                        "(for example hefx_poly_mul with HEFX_PATH_TENSOR) before using the no-allocation variant");
    }
    const size_t words = batch * p->nlimbs * (size_t)p->n;
    if (words > noalloc_scratch_words())
        return fail(ctx, HEFX_EINVAL,
                    "batch * nlimbs * N = %zu residues exceeds the %zu-residue static workspace of "
                    "hefx_poly_mul_noalloc; split the batch",
                    words, noalloc_scratch_words());
    if (batch == 0) return HEFX_OK;
    cudaError_t e = polymul_tc_noalloc(p, a, b, c, batch, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_poly_mul_noalloc");
    return HEFX_OK;
}

hefx_status hefx_stream_check(hefx_ctx* ctx, const hefx_params* p, void* stream) {
    if (!ctx) return HEFX_EINVAL;
    if (!p || p->ctx != ctx) return fail(ctx, HEFX_EINVAL, "params is null or belongs to another context");
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    uint32_t code = 0, code2 = 0;
    cudaError_t e = tc_check(p, (cudaStream_t)stream, &code);
    if (e == cudaSuccess && tc2_err(p)) {
        e = cudaMemcpyAsync(&code2, tc2_err(p), 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e == cudaSuccess && code2) e = cudaMemsetAsync(tc2_err(p), 0, 4, (cudaStream_t)stream);
        if (!code) code = code2;
    }
    if (e == cudaSuccess && p->d_err_cc) {
        uint32_t code3 = 0;
        e = cudaMemcpyAsync(&code3, p->d_err_cc, 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e == cudaSuccess && code3) e = cudaMemsetAsync(p->d_err_cc, 0, 4, (cudaStream_t)stream);
        if (!code) code = code3;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_stream_check");
    if (code) return fail(ctx, HEFX_ETIMEOUT, "a bounded device wait expired (code %u); results are invalid", code);
    return HEFX_OK;
}

hefx_status hefx_params_set_tensor_config(hefx_params* p, uint32_t log2r, uint32_t log2r2, uint32_t tile_outputs) {
    if (!p) return HEFX_EINVAL;
    const uint32_t logn = p->log2n;
    if (log2r == 0) log2r = logn / 2;
    if (log2r2 == 0) {
        const uint32_t logc = logn >= log2r ? logn - log2r : 0;
        if (log2r < 6 || log2r > 8 || logc < 6 || logc > 8)
            return fail(p->ctx, HEFX_EINVAL,
                        "tensor split 2^%u x 2^%u of N = 2^%u: both factors must be 64 .. 256 (the transposing "
                        "digit split takes 64-wide tiles; exact fp32 sums need reduction lengths <= 256)",
                        log2r, logc, logn);
    } else {
        const int log3 = (int)logn - (int)log2r - (int)log2r2;
        if (log2r < 6 || log2r > 8 || log2r2 < 4 || log2r2 > 8 || log3 < 4 || log3 > 8)
            return fail(p->ctx, HEFX_EINVAL,
                        "tensor split 2^%u x 2^%u x 2^%d of N = 2^%u: the first factor must be 64 .. 256 (the "
                        "transposing digit split takes 64-wide tiles), the others 16 .. 256 (one 64-digit "
                        "K stage at least; exact fp32 sums need reduction lengths <= 256)",
                        log2r, log2r2, log3, logn);
    }
    if (tile_outputs != 32 && tile_outputs != 64)
        return fail(p->ctx, HEFX_EINVAL, "tile_outputs must be 32 or 64, not %u", tile_outputs);
    if (tc2_wide(p) && (log2r > 6 || log2r2 > 6 || (int)logn - (int)log2r - (int)log2r2 > 6))
        return fail(p->ctx, HEFX_EUNSUPPORTED,
                    "moduli of 29-30 bits take 8-bit digits, whose fp32 sums are exact for reduction lengths "
                    "<= 64 only: every factor <= 64 (64 x 64 at N = 2^12, 64 x 32 x 32 at N = 2^16)");
    hefx_status st = use_device(p->ctx);
    if (st != HEFX_OK) return st;
    std::lock_guard<std::mutex> g(p->tc_mu);
    const uint32_t cur = p->tc_log2r ? p->tc_log2r : logn / 2;
    if (p->tc2 && (cur != log2r || p->tc_log2r2 != log2r2)) {
        // the pipelined tables are built for one split: drop them (after the device is idle)
        // so that the next tensor-path call builds the new ones
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(p->ctx, e, "hefx_params_set_tensor_config");
        tc2_free(p);
    }
    p->tc_log2r = log2r;
    p->tc_log2r2 = log2r2;
    p->tc_tile = (int)tile_outputs;
    return HEFX_OK;
}

hefx_status hefx_wait_check(hefx_ctx* ctx, const hefx_params* p, uint64_t limit_ns, int arrive, void* stream) {
    if (!ctx) return HEFX_EINVAL;
    if (!p || p->ctx != ctx) return fail(ctx, HEFX_EINVAL, "params is null or belongs to another context");
    if (limit_ns > 2000000000ull) return fail(ctx, HEFX_EINVAL, "limit_ns above the 2 s wait limit of the kernels");
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    cudaError_t e = launch_wait_check(p->d_err_cc, limit_ns, arrive, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_wait_check launch");
    return HEFX_OK;
}

hefx_status hefx_params_set_reduction(hefx_params* p, hefx_reduction ntt_red, hefx_reduction vec_red) {
    if (!p) return HEFX_EINVAL;
    if (ntt_red < HEFX_RED_SHOUP || ntt_red > HEFX_RED_BARRETT)
        return fail(p->ctx, HEFX_EINVAL, "unknown NTT reduction %d", (int)ntt_red);
    if (vec_red != HEFX_RED_MONTGOMERY && vec_red != HEFX_RED_BARRETT && vec_red != HEFX_RED_BAT_LAZY)
        return fail(p->ctx, HEFX_EINVAL, "VecModMul reduction must be Montgomery, Barrett or BAT lazy");
    if (vec_red == HEFX_RED_BAT_LAZY && p->log2n < 9)
        return fail(p->ctx, HEFX_EUNSUPPORTED, "BAT lazy reduction needs log2n >= 9");
    hefx_status st = use_device(p->ctx);
    if (st != HEFX_OK) return st;
    if (ntt_red == HEFX_RED_MONTGOMERY && !p->d_tw_fwd_mont) {
        const size_t bytes = sizeof(uint2) * (size_t)p->nlimbs * p->n;
        cudaError_t e = cudaMalloc(&p->d_tw_fwd_mont, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_tw_inv_mont, bytes);
        if (e == cudaSuccess) e = make_mont_twiddles(p, p->d_tw_fwd, p->d_tw_fwd_mont);
        if (e == cudaSuccess) e = make_mont_twiddles(p, p->d_tw_inv, p->d_tw_inv_mont);
        if (e != cudaSuccess) {
            cudaFree(p->d_tw_fwd_mont);
            cudaFree(p->d_tw_inv_mont);
            p->d_tw_fwd_mont = p->d_tw_inv_mont = nullptr;
            return cuda_fail(p->ctx, e, "Montgomery twiddle tables");
        }
    }
    p->red_ntt = ntt_red;
    p->red_vec = vec_red;
    return HEFX_OK;
}

hefx_status hefx_params_set_cc_schedule(hefx_params* p, hefx_cc_schedule schedule) {
    if (!p) return HEFX_EINVAL;
    if (schedule != HEFX_CC_AUTO && schedule != HEFX_CC_CLUSTER && schedule != HEFX_CC_TWO_PASS)
        return fail(p->ctx, HEFX_EINVAL, "unknown CUDA-core schedule %d", (int)schedule);
    if (schedule == HEFX_CC_TWO_PASS && !p->d_tw2_fwd)
        return fail(p->ctx, HEFX_EUNSUPPORTED, "the two-pass schedule is built for N = 2^16 only");
    p->cc_schedule = (int)schedule;
    return HEFX_OK;
}

/* Tuner hook: records the path AUTO resolves to. */
hefx_status hefx_params_set_auto_path(hefx_params* p, hefx_path path) {
    if (!p || (path != HEFX_PATH_CUDACORE && path != HEFX_PATH_TENSOR && path != HEFX_PATH_AUTO)) return HEFX_EINVAL;
    p->tuned_path = path;
    return HEFX_OK;
}

hefx_status hefx_mult_plan_create(hefx_ctx* ctx, const hefx_params* pq, const hefx_params* pp,
                                  const hefx_bconv_plan* bc, const uint32_t* d_kq0, const uint32_t* d_kq1,
                                  const uint32_t* d_kp0, const uint32_t* d_kp1, hefx_mult_plan** out) {
    if (!ctx || !out) return HEFX_EINVAL;
    *out = nullptr;
    if (!pq || !pp || !bc || pq->ctx != ctx || pp->ctx != ctx || bc->ctx != ctx)
        return fail(ctx, HEFX_EINVAL, "params or plan is null or belongs to another context");
    if (pq->log2n != pp->log2n || bc->log2n != pq->log2n || bc->L != pq->nlimbs || bc->Lp != pp->nlimbs)
        return fail(ctx, HEFX_EINVAL, "the conversion plan must map the Q params' limbs to the P params' limbs");
    for (uint32_t i = 0; i < pq->nlimbs; ++i)
        if (bc->src[i] != pq->primes[i]) return fail(ctx, HEFX_EINVAL, "plan source %u is not params prime %u", i, i);
    for (uint32_t j = 0; j < pp->nlimbs; ++j)
        if (bc->dst[j] != pp->primes[j]) return fail(ctx, HEFX_EINVAL, "plan target %u is not P prime %u", j, j);
    const void* keys[4] = {d_kq0, d_kq1, d_kp0, d_kp1};
    for (const void* k : keys)
        if (!k || !aligned16(k)) return fail(ctx, HEFX_EINVAL, "key pointers must be non-null and 16-byte aligned");
    hefx_mult_plan* p = new hefx_mult_plan();
    p->ctx = ctx;
    p->pq = pq;
    p->pp = pp;
    p->bc = bc;
    p->kq[0] = d_kq0;
    p->kq[1] = d_kq1;
    p->kp[0] = d_kp0;
    p->kp[1] = d_kp1;
    *out = p;
    return HEFX_OK;
}

void hefx_mult_plan_destroy(hefx_mult_plan* plan) { delete plan; }

hefx_status hefx_mult_front(hefx_ctx* ctx, const hefx_mult_plan* plan, const uint32_t* d_in, uint32_t* d_out,
                            uint32_t* d_work, void* stream) {
    if (!ctx) return HEFX_EINVAL;
    if (!plan || plan->ctx != ctx) return fail(ctx, HEFX_EINVAL, "plan is null or belongs to another context");
    if (!d_in || !d_out || !d_work || !aligned16(d_in) || !aligned16(d_out) || !aligned16(d_work))
        return fail(ctx, HEFX_EINVAL, "buffers must be non-null and 16-byte aligned");
    const size_t n = plan->pq->n, L = plan->pq->nlimbs, K = plan->pp->nlimbs;
    const size_t row = n * 4;
    const char *in = (const char*)d_in, *o = (const char*)d_out, *w = (const char*)d_work;
    auto overl = [](const char* a, size_t an, const char* b, size_t bn) { return a < b + bn && b < a + an; };
    if (overl(o, (4 * L + 2 * K) * row, in, 4 * L * row) || overl(w, (2 * L + K) * row, in, 4 * L * row) ||
        overl(w, (2 * L + K) * row, o, (4 * L + 2 * K) * row))
        return fail(ctx, HEFX_EINVAL, "d_in, d_out and d_work must not overlap");
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t *a0 = d_in, *a1 = d_in + L * n, *b0 = d_in + 2 * L * n, *b1 = d_in + 3 * L * n;
    uint32_t *d0 = d_out, *d1 = d_out + L * n, *e0q = d_out + 2 * L * n, *e1q = d_out + 3 * L * n;
    uint32_t *e0p = d_out + 4 * L * n, *e1p = d_out + (4 * L + K) * n;
    uint32_t *d2 = d_work, *c = d_work + L * n, *p = d_work + 2 * L * n;
    cudaError_t e = launch_tensor_product(plan->pq, a0, a1, b0, b1, d0, d1, d2, L, s);
    if (e == cudaSuccess) e = launch_ntt_cc(plan->pq, MODE_INV, d2, nullptr, c, L, s);  // c = INTT(d2)
    if (e == cudaSuccess)
        e = bconv_prefer_tc(plan->bc, 1) ? launch_bconv_tc(plan->bc, c, p, 1, s) : launch_bconv_cc(plan->bc, c, p, 1, s);
    if (e == cudaSuccess) e = launch_ntt_cc(plan->pp, MODE_FWD, p, nullptr, p, K, s);
    if (e == cudaSuccess) e = launch_vec_mod_mul2(plan->pq, d2, plan->kq[0], plan->kq[1], e0q, e1q, L, s);
    if (e == cudaSuccess) e = launch_vec_mod_mul2(plan->pp, p, plan->kp[0], plan->kp[1], e0p, e1p, K, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_mult_front launch");
    return HEFX_OK;
}

hefx_status hefx_mult_front_host(hefx_ctx* ctx, const hefx_mult_plan* plan, const uint32_t* h_a0,
                                 const uint32_t* h_a1, const uint32_t* h_b0, const uint32_t* h_b1, uint32_t* h_out,
                                 uint32_t* d_buf, void* stream) {
    if (!ctx) return HEFX_EINVAL;
    if (!plan || plan->ctx != ctx) return fail(ctx, HEFX_EINVAL, "plan is null or belongs to another context");
    if (!h_a0 || !h_a1 || !h_b0 || !h_b1 || !h_out || !d_buf || !aligned16(d_buf))
        return fail(ctx, HEFX_EINVAL, "null host buffer or null / misaligned device buffer");
    hefx_status st = use_device(ctx);
    if (st != HEFX_OK) return st;
    const size_t n = plan->pq->n, L = plan->pq->nlimbs, K = plan->pp->nlimbs;
    const size_t in_bytes = L * n * 4;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *d_in = d_buf, *d_out = d_buf + 4 * L * n, *d_work = d_buf + (8 * L + 2 * K) * n;
    const uint32_t* h_in[4] = {h_a0, h_a1, h_b0, h_b1};
    cudaError_t e = cudaSuccess;
    const ptrdiff_t gap = h_a1 - h_a0;  // equally spaced inputs: one pitched copy instead of four
    if (gap >= (ptrdiff_t)(L * n) && h_b0 - h_a1 == gap && h_b1 - h_b0 == gap)
        e = cudaMemcpy2DAsync(d_in, in_bytes, h_a0, (size_t)gap * 4, in_bytes, 4, cudaMemcpyHostToDevice, s);
    else
        for (int i = 0; i < 4 && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(d_in + i * L * n, h_in[i], in_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_mult_front_host input copy");
    st = hefx_mult_front(ctx, plan, d_in, d_out, d_work, stream);
    if (st != HEFX_OK) return st;
    e = cudaMemcpyAsync(h_out, d_out, (4 * L + 2 * K) * n * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hefx_mult_front_host output copy");
    return HEFX_OK;
}

}  // extern "C"
