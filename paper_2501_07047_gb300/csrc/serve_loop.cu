// Native serving loop (hefx_serve_run): continuous batching of HE-Mult front-half requests on
// device-resident ciphertexts, the request loop of serve.py without its interpreter overhead.
// Real-time arrivals, FIFO admission against a device-memory budget and a pool of result
// slots (head-of-line blocking), the requests admitted in one pass grouped by ring degree and
// P parameter set into shared launches (mult_front_batch_dev: five launches per group),
// groups round-robin over the caller's streams, completion by one event per group (a stream
// completes its groups in order, so only the oldest group of each stream is polled).
#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <thread>
#include <utility>
#include <vector>

#include "hefx_internal.h"

using namespace hefx;

namespace {

struct Group {
    cudaEvent_t ev;
    std::vector<size_t> reqs;
};

hefx_status fail_sv(hefx_ctx* ctx, hefx_status st, const char* msg) {
    if (ctx) {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->last_error = msg;
    }
    return st;
}

}  // namespace

extern "C" hefx_status hefx_serve_run(hefx_ctx* ctx, hefx_mult_batch* batch, const hefx_serve_request* reqs,
                                      size_t n, const hefx_serve_config* cfg, hefx_serve_result* out) {
    if (!ctx) return HEFX_EINVAL;
    if (!batch || !cfg || !out || (n && !reqs)) return fail_sv(ctx, HEFX_EINVAL, "hefx_serve_run: null argument");
    if (cfg->nstreams == 0 || !cfg->streams || cfg->nslots == 0 || !cfg->slot_out || !cfg->slot_work ||
        cfg->max_group == 0)
        return fail_sv(ctx, HEFX_EINVAL, "hefx_serve_run: need streams, result slots and max_group >= 1");
    for (size_t i = 0; i < n; ++i) {
        MultPlanView v;
        if (!mult_plan_view(reqs[i].plan, &v) || v.ctx != ctx)
            return fail_sv(ctx, HEFX_EINVAL, "hefx_serve_run: a request's plan is null or of another context");
        if (!reqs[i].d_a0 || !reqs[i].d_a1 || !reqs[i].d_b0 || !reqs[i].d_b1)
            return fail_sv(ctx, HEFX_EINVAL, "hefx_serve_run: null input");
        if (i && reqs[i].arrival_s < reqs[i - 1].arrival_s)
            return fail_sv(ctx, HEFX_EINVAL, "hefx_serve_run: requests must be sorted by arrival");
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail_sv(ctx, HEFX_ECUDA, "cudaSetDevice failed");
    // at most one group per slot is in flight: one event each
    std::vector<cudaEvent_t> ev_free(cfg->nslots);
    for (auto& e : ev_free)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            for (auto& x : ev_free)
                if (x) cudaEventDestroy(x);
            return fail_sv(ctx, HEFX_ECUDA, "hefx_serve_run: event creation failed");
        }
    std::vector<uint32_t> slot_free;
    for (uint32_t k = cfg->nslots; k-- > 0;) slot_free.push_back(k);
    std::vector<std::deque<Group>> flight(cfg->nstreams);
    std::deque<size_t> queue;
    for (size_t i = 0; i < n; ++i) out[i] = hefx_serve_result{-1.0, -1.0, HEFX_SERVE_PENDING, 0};

    using clock = std::chrono::steady_clock;
    const auto t0 = clock::now();
    auto now_s = [&]() { return std::chrono::duration<double>(clock::now() - t0).count(); };
    uint64_t in_use = 0, high_water = 0;
    size_t next = 0, finished = 0, active = 0, max_active = 0, groups = 0;
    uint32_t next_stream = 0;
    hefx_status st = HEFX_OK;
    std::vector<const hefx_mult_plan*> plans;
    std::vector<const uint32_t*> in[4];
    std::vector<uint32_t*> outs, works;
    while (finished < n && st == HEFX_OK) {
        bool progress = false;
        const double t = now_s();
        while (next < n && reqs[next].arrival_s <= t) {  // arrivals
            if (reqs[next].bytes > cfg->budget_bytes) {
                out[next].status = HEFX_SERVE_REJECTED;
                ++finished;
            } else {
                queue.push_back(next);
            }
            ++next;
            progress = true;
        }
        // admission (FIFO, head-of-line blocking) and grouping by (ring degree, P set)
        std::map<std::pair<uint32_t, const void*>, std::vector<size_t>> by_key;
        while (!queue.empty() && !slot_free.empty() && in_use + reqs[queue.front()].bytes <= cfg->budget_bytes) {
            const size_t i = queue.front();
            queue.pop_front();
            in_use += reqs[i].bytes;
            high_water = std::max(high_water, in_use);
            out[i].slot = slot_free.back();
            slot_free.pop_back();
            out[i].admitted_s = now_s();
            out[i].status = HEFX_SERVE_RUNNING;
            MultPlanView v;
            mult_plan_view(reqs[i].plan, &v);
            by_key[{v.pq->log2n, (const void*)v.pp}].push_back(i);
            ++active;
        }
        max_active = std::max(max_active, active);
        for (auto& kv : by_key) {
            const std::vector<size_t>& ids = kv.second;
            for (size_t g0 = 0; g0 < ids.size() && st == HEFX_OK; g0 += cfg->max_group) {
                const size_t g1 = std::min(ids.size(), g0 + (size_t)cfg->max_group);
                plans.clear();
                outs.clear();
                works.clear();
                for (auto& v : in) v.clear();
                Group grp;
                for (size_t k = g0; k < g1; ++k) {
                    const hefx_serve_request& r = reqs[ids[k]];
                    plans.push_back(r.plan);
                    in[0].push_back(r.d_a0);
                    in[1].push_back(r.d_a1);
                    in[2].push_back(r.d_b0);
                    in[3].push_back(r.d_b1);
                    outs.push_back(cfg->slot_out[out[ids[k]].slot]);
                    works.push_back(cfg->slot_work[out[ids[k]].slot]);
                    grp.reqs.push_back(ids[k]);
                }
                const uint32_t si = next_stream;
                next_stream = (next_stream + 1) % cfg->nstreams;
                cudaStream_t s = (cudaStream_t)cfg->streams[si];
                const uint32_t* const* const inputs[4] = {in[0].data(), in[1].data(), in[2].data(), in[3].data()};
                st = mult_front_batch_dev(ctx, batch, plans.data(), (uint32_t)plans.size(), inputs, outs.data(),
                                          works.data(), s);
                if (st != HEFX_OK) break;
                grp.ev = ev_free.back();  // one group per admitted slot at most, so never empty
                ev_free.pop_back();
                if (cudaEventRecord(grp.ev, s) != cudaSuccess) {
                    st = fail_sv(ctx, HEFX_ECUDA, "hefx_serve_run: event record failed");
                    break;
                }
                flight[si].push_back(std::move(grp));
                ++groups;
            }
            progress = true;
        }
        // completions: the oldest group of each stream
        for (auto& q : flight) {
            while (!q.empty() && st == HEFX_OK) {
                const cudaError_t e = cudaEventQuery(q.front().ev);
                if (e == cudaErrorNotReady) break;
                if (e != cudaSuccess) {
                    st = fail_sv(ctx, HEFX_ECUDA, cudaGetErrorString(e));
                    break;
                }
                const double tc = now_s();
                for (size_t i : q.front().reqs) {
                    out[i].completed_s = tc;
                    out[i].status = HEFX_SERVE_DONE;
                    in_use -= reqs[i].bytes;
                    slot_free.push_back(out[i].slot);
                    --active;
                    ++finished;
                }
                ev_free.push_back(q.front().ev);
                q.pop_front();
                progress = true;
            }
        }
        if (!progress) {
            if (active == 0 && queue.empty() && next < n) {  // idle until the next arrival
                const double wait = reqs[next].arrival_s - now_s();
                if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 1e-3) - 1e-4));
            } else {
                std::this_thread::yield();
            }
        }
    }
    // on an error, wait for what was launched before releasing the events
    for (auto& q : flight)
        for (auto& g : q) {
            cudaEventSynchronize(g.ev);
            ev_free.push_back(g.ev);
        }
    for (auto& e : ev_free) cudaEventDestroy(e);
    if (cfg->stats) {
        cfg->stats->max_active = max_active;
        cfg->stats->memory_high_water_bytes = high_water;
        cfg->stats->groups = groups;
    }
    return st;
}
