// Batched serving request: the HE-Mult front half (hefx_mult_front) of several ciphertext
// pairs of one ring degree in shared launches.  Requests may differ in limb count (each brings
// its own parameter sets and conversion plan); every stage runs once over the rows of all of
// them: the tensor product and the key products as row lists, INTT(d2) and NTT over P as
// row-list transforms, the conversion to P as a list launch with one block row per request.
// Per request only the input upload and the output read-back remain.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hefx_internal.h"
#include "modarith.cuh"

namespace hefx {
namespace {

// One limb row of an elementwise stage: x = (a0, a1, b0, b1) -> y = (d0, d1, d2) for the tensor
// product; x = (src, key0, key1) -> y = (e0, e1) for the key products.
struct MultRow {
    const uint32_t* x[4];
    uint32_t* y[3];
    const LimbConst* lc;
};
static_assert(sizeof(MultRow) == 64, "MultRow is one 64-byte line");

__device__ __forceinline__ uint32_t mulmod_r(uint32_t x, uint32_t y, const LimbConst& c) {
    const uint32_t t = mul_mont_lazy(x, y, c.q, c.qinv_neg);
    return csub(mul_mont_lazy(t, c.r2, c.q, c.qinv_neg), c.q);
}
__device__ __forceinline__ uint32_t mac2_r(uint32_t a, uint32_t b, uint32_t c2, uint32_t d, const LimbConst& k) {
    const uint32_t t = mul_mont_lazy(a, b, k.q, k.qinv_neg) + mul_mont_lazy(c2, d, k.q, k.qinv_neg);
    return csub(mul_mont_lazy(t, k.r2, k.q, k.qinv_neg), k.q);
}

// grid-stride over (row, 16-byte group) of every row; n4 = N / 4 groups per row
__global__ void __launch_bounds__(256) tp_rows_kernel(const MultRow* __restrict__ rows, uint32_t nrows, uint32_t log2n4) {
    griddep_wait();
    const size_t total = (size_t)nrows << log2n4;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const MultRow& r = rows[i >> log2n4];
        const size_t e = i & (((size_t)1 << log2n4) - 1);
        const LimbConst c = *r.lc;
        const uint4 x0 = reinterpret_cast<const uint4*>(r.x[0])[e], x1 = reinterpret_cast<const uint4*>(r.x[1])[e];
        const uint4 y0 = reinterpret_cast<const uint4*>(r.x[2])[e], y1 = reinterpret_cast<const uint4*>(r.x[3])[e];
        reinterpret_cast<uint4*>(r.y[0])[e] = make_uint4(mulmod_r(x0.x, y0.x, c), mulmod_r(x0.y, y0.y, c),
                                                         mulmod_r(x0.z, y0.z, c), mulmod_r(x0.w, y0.w, c));
        reinterpret_cast<uint4*>(r.y[1])[e] =
            make_uint4(mac2_r(x0.x, y1.x, x1.x, y0.x, c), mac2_r(x0.y, y1.y, x1.y, y0.y, c),
                       mac2_r(x0.z, y1.z, x1.z, y0.z, c), mac2_r(x0.w, y1.w, x1.w, y0.w, c));
        reinterpret_cast<uint4*>(r.y[2])[e] = make_uint4(mulmod_r(x1.x, y1.x, c), mulmod_r(x1.y, y1.y, c),
                                                         mulmod_r(x1.z, y1.z, c), mulmod_r(x1.w, y1.w, c));
    }
}

__global__ void __launch_bounds__(256) km_rows_kernel(const MultRow* __restrict__ rows, uint32_t nrows, uint32_t log2n4) {
    griddep_wait();
    const size_t total = (size_t)nrows << log2n4;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const MultRow& r = rows[i >> log2n4];
        const size_t e = i & (((size_t)1 << log2n4) - 1);
        const LimbConst c = *r.lc;
        const uint4 a = reinterpret_cast<const uint4*>(r.x[0])[e];
        const uint4 k0 = reinterpret_cast<const uint4*>(r.x[1])[e], k1 = reinterpret_cast<const uint4*>(r.x[2])[e];
        reinterpret_cast<uint4*>(r.y[0])[e] = make_uint4(mulmod_r(a.x, k0.x, c), mulmod_r(a.y, k0.y, c),
                                                         mulmod_r(a.z, k0.z, c), mulmod_r(a.w, k0.w, c));
        reinterpret_cast<uint4*>(r.y[1])[e] = make_uint4(mulmod_r(a.x, k1.x, c), mulmod_r(a.y, k1.y, c),
                                                         mulmod_r(a.z, k1.z, c), mulmod_r(a.w, k1.w, c));
    }
}

unsigned grid_for(size_t groups) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (unsigned)std::max<size_t>(1, std::min<size_t>((groups + 255) / 256, (size_t)sms * 8));
}

}  // namespace
}  // namespace hefx

using namespace hefx;

// Descriptor staging of batched requests: a ring of slots, each a pinned host area and a
// device area of the same size; a slot is reused once the event recorded after its launches
// has completed.
struct hefx_mult_batch {
    hefx_ctx* ctx = nullptr;
    uint32_t max_requests = 0, max_rows = 0;
    size_t slot_bytes = 0;
    static constexpr int kSlots = 64;
    uint8_t* host[kSlots] = {};
    uint8_t* dev[kSlots] = {};
    cudaEvent_t ev[kSlots] = {};
    bool used[kSlots] = {};
    int next = 0;
};

namespace {

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets of the descriptor arrays inside a slot for R1 Q rows, count requests, K P limbs
struct Layout {
    size_t tp, intt, bc, nttp, km, total;
};
Layout layout(size_t r1, size_t count, size_t K) {
    Layout l;
    l.tp = 0;
    l.intt = align_up(l.tp + r1 * sizeof(MultRow));
    l.bc = align_up(l.intt + r1 * sizeof(RowDesc));
    l.nttp = align_up(l.bc + count * sizeof(BcListEntry));
    l.km = align_up(l.nttp + count * K * sizeof(RowDesc));
    l.total = align_up(l.km + (r1 + count * K) * sizeof(MultRow));
    return l;
}

RowDesc rowdesc(const hefx_params* p, uint32_t l, const uint32_t* in, uint32_t* out) {
    RowDesc r;
    memset(&r, 0, sizeof r);
    r.in = in;
    r.out = out;
    r.lc = p->d_lc + l;
    r.twf = p->d_tw_fwd + (size_t)l * p->n;
    r.twi = p->d_tw_inv + (size_t)l * p->n;
    r.limb = l;
    return r;
}

hefx_status fail_mb(hefx_ctx* ctx, hefx_status st, const char* fmt, ...) {
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

}  // namespace

extern "C" {

hefx_status hefx_mult_batch_create(hefx_ctx* ctx, uint32_t max_requests, uint32_t max_limbs, hefx_mult_batch** out) {
    if (!ctx || !out) return HEFX_EINVAL;
    *out = nullptr;
    if (max_requests == 0 || max_requests > 1024 || max_limbs == 0 || max_limbs > 4096)
        return fail_mb(ctx, HEFX_EINVAL, "hefx_mult_batch_create: need 1..1024 requests of 1..4096 limbs");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail_mb(ctx, HEFX_ECUDA, "cudaSetDevice failed");
    hefx_mult_batch* mb = new hefx_mult_batch();
    mb->ctx = ctx;
    mb->max_requests = max_requests;
    mb->max_rows = max_limbs;
    const size_t K = 64;  // room for up to 64 special limbs per request
    mb->slot_bytes = layout((size_t)max_requests * max_limbs, max_requests, K).total;
    // the slots are the in-flight limit of batched calls: a call waits only when all of them
    // are still read by launches
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < hefx_mult_batch::kSlots && e == cudaSuccess; ++s) {
        e = cudaMallocHost(&mb->host[s], mb->slot_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&mb->dev[s], mb->slot_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&mb->ev[s], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        hefx_mult_batch_destroy(mb);
        return fail_mb(ctx, HEFX_ENOMEM, "hefx_mult_batch_create: allocation failed");
    }
    *out = mb;
    return HEFX_OK;
}

void hefx_mult_batch_destroy(hefx_mult_batch* mb) {
    if (!mb) return;
    for (int s = 0; s < hefx_mult_batch::kSlots; ++s) {
        if (mb->ev[s]) {
            cudaEventSynchronize(mb->ev[s]);
            cudaEventDestroy(mb->ev[s]);
        }
        if (mb->dev[s]) cudaFree(mb->dev[s]);
        if (mb->host[s]) cudaFreeHost(mb->host[s]);
    }
    delete mb;
}

}  // extern "C"

namespace {

bool overlap_bytes(const void* a, size_t an, const void* b, size_t bn) {
    const char *x = (const char*)a, *y = (const char*)b;
    return x < y + bn && y < x + an;
}

// Body of both batched calls: validation, the descriptors and the five shared launches.
// inputs[i][r] is request r's input i (a0, a1, b0, b1; [L_r][N] on the device), d_out[r] its
// [4 L_r + 2K][N] outputs, d_work[r] its [2 L_r + K][N] workspace.  With host copies, each
// request's inputs are first uploaded from hin[i][r] into inputs[i][r], and its outputs are
// read back into h_out[r] after the launches.
hefx_status front_batch(hefx_ctx* ctx, hefx_mult_batch* mb, const hefx_mult_plan* const* plans, uint32_t count,
                        const uint32_t* const* const inputs[4], uint32_t* const* d_out, uint32_t* const* d_work,
                        const uint32_t* const* const hin[4], uint32_t* const* h_out, cudaStream_t s,
                        const char* name) {
    if (!ctx) return HEFX_EINVAL;
    if (!mb || mb->ctx != ctx) return fail_mb(ctx, HEFX_EINVAL, "batch object is null or of another context");
    if (count == 0) return HEFX_OK;
    const bool host = hin != nullptr;
    if (count > mb->max_requests || !plans || !inputs[0] || !inputs[1] || !inputs[2] || !inputs[3] || !d_out ||
        !d_work || (host && (!hin[0] || !hin[1] || !hin[2] || !hin[3] || !h_out)))
        return fail_mb(ctx, HEFX_EINVAL, "%s: count above the batch object's or null arrays", name);
    MultPlanView v0;
    if (!mult_plan_view(plans[0], &v0) || v0.ctx != ctx)
        return fail_mb(ctx, HEFX_EINVAL, "%s: plan 0 is null or of another context", name);
    const uint32_t K = v0.pp->nlimbs, logn = v0.pp->log2n;
    const size_t n = (size_t)1 << logn;
    size_t r1 = 0;
    for (uint32_t r = 0; r < count; ++r) {
        MultPlanView v;
        if (!mult_plan_view(plans[r], &v) || v.ctx != ctx)
            return fail_mb(ctx, HEFX_EINVAL, "%s: a plan is null or of another context", name);
        if (v.pq->log2n != v0.pq->log2n || v.pp != v0.pp)
            return fail_mb(ctx, HEFX_EINVAL, "%s: every request of a batch shares the ring degree and P", name);
        if (v.pq->nlimbs > mb->max_rows)
            return fail_mb(ctx, HEFX_EINVAL, "%s: more limbs than the batch object holds", name);
        const size_t L = v.pq->nlimbs;
        const void* bufs[6] = {inputs[0][r], inputs[1][r], inputs[2][r], inputs[3][r], d_out[r], d_work[r]};
        const size_t sizes[6] = {L * n * 4, L * n * 4, L * n * 4, L * n * 4, (4 * L + 2 * K) * n * 4,
                                 (2 * L + K) * n * 4};
        for (int i = 0; i < 6; ++i)
            if (!bufs[i] || ((uintptr_t)bufs[i] & 15))
                return fail_mb(ctx, HEFX_EINVAL, "%s: null or misaligned device buffer", name);
        // the outputs and the workspace are written: neither may overlap any buffer of the request
        for (int w = 4; w < 6; ++w)
            for (int i = 0; i < 6; ++i)
                if (i != w && overlap_bytes(bufs[w], sizes[w], bufs[i], sizes[i]))
                    return fail_mb(ctx, HEFX_EINVAL, "%s: a request's output or workspace overlaps its other buffers",
                                   name);
        if (host && (!hin[0][r] || !hin[1][r] || !hin[2][r] || !hin[3][r] || !h_out[r]))
            return fail_mb(ctx, HEFX_EINVAL, "%s: null host buffer", name);
        r1 += L;
    }
    const hefx_params* pp = v0.pp;
    if (K > 64) return fail_mb(ctx, HEFX_EUNSUPPORTED, "%s: at most 64 special limbs", name);
    const Layout lay = layout(r1, count, K);
    if (lay.total > mb->slot_bytes) return fail_mb(ctx, HEFX_EINVAL, "%s: batch too large", name);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail_mb(ctx, HEFX_ECUDA, "cudaSetDevice failed");
    const int slot = mb->next;
    mb->next = (mb->next + 1) % hefx_mult_batch::kSlots;
    if (mb->used[slot] && cudaEventSynchronize(mb->ev[slot]) != cudaSuccess)
        return fail_mb(ctx, HEFX_ECUDA, "%s: waiting for a descriptor slot failed", name);
    uint8_t* hb = mb->host[slot];
    uint8_t* db = mb->dev[slot];
    MultRow* tp = reinterpret_cast<MultRow*>(hb + lay.tp);
    RowDesc* intt = reinterpret_cast<RowDesc*>(hb + lay.intt);
    BcListEntry* bc = reinterpret_cast<BcListEntry*>(hb + lay.bc);
    RowDesc* nttp = reinterpret_cast<RowDesc*>(hb + lay.nttp);
    MultRow* km = reinterpret_cast<MultRow*>(hb + lay.km);
    size_t q = 0, kmi = 0;
    uint32_t lp_max = 0;
    cudaError_t e = cudaSuccess;
    for (uint32_t r = 0; r < count && e == cudaSuccess; ++r) {
        MultPlanView v;
        mult_plan_view(plans[r], &v);
        const size_t L = v.pq->nlimbs;
        // workspace: d2 (L rows) | c = INTT(d2) (L) | p (K)
        uint32_t* out = d_out[r];
        uint32_t* d2 = d_work[r];
        uint32_t* c = d2 + L * n;
        uint32_t* pr = c + L * n;
        if (host) {
            const size_t in_bytes = L * n * 4;
            const bool packed = inputs[1][r] == inputs[0][r] + L * n && inputs[2][r] == inputs[1][r] + L * n &&
                                inputs[3][r] == inputs[2][r] + L * n;
            const ptrdiff_t gap = hin[1][r] - hin[0][r];
            if (packed && gap >= (ptrdiff_t)(L * n) && hin[2][r] - hin[1][r] == gap && hin[3][r] - hin[2][r] == gap)
                e = cudaMemcpy2DAsync(const_cast<uint32_t*>(inputs[0][r]), in_bytes, hin[0][r], (size_t)gap * 4,
                                      in_bytes, 4, cudaMemcpyHostToDevice, s);
            else
                for (int i = 0; i < 4 && e == cudaSuccess; ++i)
                    e = cudaMemcpyAsync(const_cast<uint32_t*>(inputs[i][r]), hin[i][r], in_bytes,
                                        cudaMemcpyHostToDevice, s);
        }
        for (uint32_t l = 0; l < L; ++l, ++q) {
            MultRow& t = tp[q];
            for (int i = 0; i < 4; ++i) t.x[i] = inputs[i][r] + l * n;
            t.y[0] = out + l * n;
            t.y[1] = out + (L + l) * n;
            t.y[2] = d2 + l * n;
            t.lc = v.pq->d_lc + l;
            intt[q] = rowdesc(v.pq, l, d2 + l * n, c + l * n);
            MultRow& k = km[kmi++];
            memset(&k, 0, sizeof k);
            k.x[0] = d2 + l * n;
            k.x[1] = v.kq[0] + l * n;
            k.x[2] = v.kq[1] + l * n;
            k.y[0] = out + (2 * L + l) * n;
            k.y[1] = out + (3 * L + l) * n;
            k.lc = v.pq->d_lc + l;
        }
        bc[r].c = v.bc->d_const;
        bc[r].in = c;
        bc[r].out = pr;
        lp_max = std::max(lp_max, v.bc->Lp);
        for (uint32_t j = 0; j < K; ++j) {
            nttp[(size_t)r * K + j] = rowdesc(pp, j, pr + j * n, pr + j * n);
            MultRow& k = km[kmi++];
            memset(&k, 0, sizeof k);
            k.x[0] = pr + j * n;
            k.x[1] = v.kp[0] + j * n;
            k.x[2] = v.kp[1] + j * n;
            k.y[0] = out + (4 * L + j) * n;
            k.y[1] = out + (4 * L + K + j) * n;
            k.lc = pp->d_lc + j;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(db, hb, lay.total, cudaMemcpyHostToDevice, s);
    const uint32_t log2n4 = logn - 2;
    const size_t nkm = r1 + (size_t)count * K;
    if (e == cudaSuccess) {
        tp_rows_kernel<<<grid_for(r1 << log2n4), 256, 0, s>>>(reinterpret_cast<const MultRow*>(db + lay.tp),
                                                              (uint32_t)r1, log2n4);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = launch_ntt_cc_rows(v0.pq, MODE_INV, reinterpret_cast<const RowDesc*>(db + lay.intt), r1, s);
    if (e == cudaSuccess)
        e = launch_bconv_cc_list(reinterpret_cast<const BcListEntry*>(db + lay.bc), count, logn, lp_max, s);
    if (e == cudaSuccess)
        e = launch_ntt_cc_rows(pp, MODE_FWD, reinterpret_cast<const RowDesc*>(db + lay.nttp), (size_t)count * K, s);
    if (e == cudaSuccess) {
        km_rows_kernel<<<grid_for(nkm << log2n4), 256, 0, s>>>(reinterpret_cast<const MultRow*>(db + lay.km),
                                                               (uint32_t)nkm, log2n4);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(mb->ev[slot], s);  // the slot's descriptors are free after this
    mb->used[slot] = true;
    for (uint32_t r = 0; host && r < count && e == cudaSuccess; ++r) {
        MultPlanView v;
        mult_plan_view(plans[r], &v);
        const size_t L = v.pq->nlimbs;
        e = cudaMemcpyAsync(h_out[r], d_out[r], (4 * L + 2 * K) * n * 4, cudaMemcpyDeviceToHost, s);
    }
    if (e != cudaSuccess) return fail_mb(ctx, HEFX_ECUDA, "%s", cudaGetErrorString(e));
    return HEFX_OK;
}

}  // namespace

hefx_status hefx::mult_front_batch_dev(hefx_ctx* ctx, hefx_mult_batch* mb, const hefx_mult_plan* const* plans,
                                       uint32_t count, const uint32_t* const* const inputs[4],
                                       uint32_t* const* d_out, uint32_t* const* d_work, cudaStream_t s) {
    return front_batch(ctx, mb, plans, count, inputs, d_out, d_work, nullptr, nullptr, s, "hefx_serve_run");
}

extern "C" {

hefx_status hefx_mult_front_batch_host(hefx_ctx* ctx, hefx_mult_batch* mb, const hefx_mult_plan* const* plans,
                                       uint32_t count, const uint32_t* const* h_a0, const uint32_t* const* h_a1,
                                       const uint32_t* const* h_b0, const uint32_t* const* h_b1,
                                       uint32_t* const* h_out, uint32_t* const* d_buf, void* stream) {
    if (!ctx) return HEFX_EINVAL;
    if (count == 0) return HEFX_OK;
    if (!mb || mb->ctx != ctx) return fail_mb(ctx, HEFX_EINVAL, "batch object is null or of another context");
    if (count > mb->max_requests || !plans || !d_buf)
        return fail_mb(ctx, HEFX_EINVAL, "hefx_mult_front_batch_host: count above the batch object's or null arrays");
    // each d_buf[r]: inputs (4L rows) | outputs (4L + 2K rows) | workspace (2L + K rows)
    std::vector<const uint32_t*> in[4];
    std::vector<uint32_t*> out(count), work(count);
    for (uint32_t r = 0; r < count; ++r) {
        MultPlanView v;
        if (!mult_plan_view(plans[r], &v) || v.ctx != ctx || !d_buf[r])
            return fail_mb(ctx, HEFX_EINVAL, "hefx_mult_front_batch_host: a plan or buffer is null or foreign");
        const size_t L = v.pq->nlimbs, K = v.pp->nlimbs, n = (size_t)v.pq->n;
        for (int i = 0; i < 4; ++i) in[i].push_back(d_buf[r] + i * L * n);
        out[r] = d_buf[r] + 4 * L * n;
        work[r] = out[r] + (4 * L + 2 * K) * n;
    }
    const uint32_t* const* const inputs[4] = {in[0].data(), in[1].data(), in[2].data(), in[3].data()};
    const uint32_t* const* const hin[4] = {h_a0, h_a1, h_b0, h_b1};
    if (!h_a0 || !h_a1 || !h_b0 || !h_b1 || !h_out)
        return fail_mb(ctx, HEFX_EINVAL, "hefx_mult_front_batch_host: null host arrays");
    return front_batch(ctx, mb, plans, count, inputs, out.data(), work.data(), hin, h_out, (cudaStream_t)stream,
                       "hefx_mult_front_batch_host");
}

hefx_status hefx_mult_front_batch(hefx_ctx* ctx, hefx_mult_batch* mb, const hefx_mult_plan* const* plans,
                                  uint32_t count, const uint32_t* const* d_a0, const uint32_t* const* d_a1,
                                  const uint32_t* const* d_b0, const uint32_t* const* d_b1, uint32_t* const* d_out,
                                  uint32_t* const* d_work, void* stream) {
    const uint32_t* const* const inputs[4] = {d_a0, d_a1, d_b0, d_b1};
    return front_batch(ctx, mb, plans, count, inputs, d_out, d_work, nullptr, nullptr, (cudaStream_t)stream,
                       "hefx_mult_front_batch");
}

}  // extern "C"
