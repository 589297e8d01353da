"""Continuous-batching server for ciphertext-multiply requests on one GPU.

A request carries two ciphertexts (a0, a1), (b0, b1) of an RNS polynomial ring (degree N,
L limbs of 28-bit primes) in evaluation form and asks for the HE-Mult front half that the
hefx kernels cover (Sec. III, HE-Mult; Sec. V-B: NTT/INTT/BConv dominate it):

    d0 = a0 o b0,  d1 = a0 o b1 + a1 o b0,  d2 = a1 o b1          (tensor product)
    c  = INTT(d2)                                                   (to coefficients)
    p  = BConv_{Q -> P}(c) over 8 special 30-bit primes, then NTT(p) (ModUp of d2)
    e_k = (d2 | p) o key_k  over the L + 8 limbs of Q u P, k = 0, 1 (key products)

and returns (d0, d1, e0, e1).  Key material is synthetic and seeded per shape.

Serving policy
 - Requests wait in arrival order.  One is admitted as soon as its device memory
   (inputs, outputs and temporaries, all device-resident while it runs) fits in the
   remaining budget and a slot is free; a request that can never fit is rejected.
 - Each admitted request is enqueued on its own CUDA stream out of a small pool, so
   requests that arrive while others are running overlap on the device.
 - Completion is observed through a CUDA event; the outputs are read back to pinned host
   memory, the request's memory returns to the budget and its latency
   (completion - arrival) is recorded.

The admission and budget logic is device-independent (`Admission`) and is tested on the
CPU; `GpuExecutor` runs the stages through the hefx C ABI.
"""
from __future__ import annotations

import collections
import dataclasses
import gc
import time

import numpy as np

from . import inputs

N_SPECIAL = 8  # auxiliary primes P of the key-switching basis


@dataclasses.dataclass
class Request:
    rid: int
    logn: int
    L: int
    arrival: float           # seconds since the start of the run
    variant: int = 0         # which pre-generated input set to use
    admitted: float = -1.0
    completed: float = -1.0
    status: str = "pending"  # pending | running | done | rejected
    outputs: tuple = ()


def request_bytes(logn: int, L: int) -> int:
    """Device bytes of one request: 4 input, 4 output and 2 temporary limb-sets over Q (the
    inputs, d0, d1, the Q parts of e0, e1, then d2 and INTT(d2)), 2 output and 1 temporary
    limb-sets over P (uint32 residues)."""
    n = 1 << logn
    return 4 * n * (10 * L + 3 * N_SPECIAL)


class Admission:
    """FIFO admission against a device-memory budget and a slot limit."""

    def __init__(self, budget_bytes: int, max_slots: int):
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.in_use = 0
        self.active = 0
        self.high_water = 0
        self.queue = collections.deque()

    def submit(self, req: Request) -> None:
        if request_bytes(req.logn, req.L) > self.budget:
            req.status = "rejected"
            return
        self.queue.append(req)

    def admit(self):
        """Yields the requests that can start now, in arrival order (head-of-line blocking)."""
        while self.queue and self.active < self.max_slots:
            need = request_bytes(self.queue[0].logn, self.queue[0].L)
            if self.in_use + need > self.budget:
                break
            req = self.queue.popleft()
            self.in_use += need
            self.active += 1
            self.high_water = max(self.high_water, self.in_use)
            req.status = "running"
            yield req

    def release(self, req: Request) -> None:
        self.in_use -= request_bytes(req.logn, req.L)
        self.active -= 1
        assert self.in_use >= 0 and self.active >= 0


class GpuExecutor:
    """Runs requests through the hefx C ABI on a pool of CUDA streams.

    grouped=False: one native call per request (`hefx_mult_front_host`, six launches each).
    grouped=True: the requests admitted together are grouped by ring degree and each group
    (at most `max_group` requests) is one `hefx_mult_front_batch_host` call whose five
    launches cover every request of the group (continuous batching across requests).
    resident=True: the requests' ciphertexts live in device memory (uploaded once, like the
    keys) and their results stay there (`hefx_mult_front_batch`), so nothing crosses the host
    link per request; `outputs` reads a result back only when asked."""

    def __init__(self, ctx: int, nstreams: int = 8, seed: int = 5, variants: int = 2, slots: int | None = None,
                 grouped: bool = False, max_group: int = 32, resident: bool = False):
        import torch

        from . import hefx
        self.torch, self.hefx = torch, hefx
        self.ctx = ctx
        self.streams = [torch.cuda.Stream() for _ in range(nstreams)]
        self.next_stream = 0
        self.seed = seed
        self.variants = variants
        self.shapes = {}
        self.pools = {}
        self.pparams_cache = {}
        self.qprimes = inputs.source_primes(36)
        self.free_slots = []
        # the serving loop keeps at most 4 requests per stream in flight: allocate their slots
        # now (pinned host memory is slow to allocate while requests are being served)
        self.free_slots = [self._slot() for _ in range(4 * nstreams if slots is None else slots)]
        self.pprimes = inputs.special_primes(N_SPECIAL)
        self.grouped = grouped
        self.resident = resident
        self.max_group = max_group
        self.batch = hefx.hefx_mult_batch_create(ctx, max_group if grouped else 1, len(self.qprimes)) \
            if grouped or resident else None

    # ---------------------------------------------------------------- per-shape resources
    def pool(self, logn: int):
        """Inputs and keys for ring degree N over all 36 Q limbs (+ 8 P limbs); a request with
        L limbs uses the first L rows, which are uniform residues of q_0 .. q_{L-1}."""
        if logn in self.pools:
            return self.pools[logn]
        torch = self.torch
        n, LQ = 1 << logn, len(self.qprimes)
        ks = inputs.derive_seed(self.seed, 1000, logn)

        def dev(arr):
            return torch.from_numpy(np.ascontiguousarray(arr).view(np.int32).copy()).cuda()

        pl = {
            "kQ": [dev(inputs.residue_tensor(inputs.derive_seed(ks, k, 0), 1, self.qprimes, n)[0]) for k in range(2)],
            "kP": [dev(inputs.residue_tensor(inputs.derive_seed(ks, k, 1), 1, self.pprimes, n)[0]) for k in range(2)],
            "host_in": [],
        }
        for v in range(self.variants):
            sv = inputs.derive_seed(self.seed, 2000, logn, v)
            arrs = [inputs.residue_tensor(inputs.derive_seed(sv, c), 1, self.qprimes, n)[0] for c in range(4)]
            # one pinned block [4][36][N]: a request's four inputs are equally spaced, which the
            # native call uploads as one pitched copy
            block = torch.from_numpy(np.stack(arrs).view(np.int32).copy()).pin_memory()
            pl["host_in"].append([block[c] for c in range(4)])
            if self.resident:  # the same ciphertexts, resident in device memory
                dblock = block.cuda()
                pl.setdefault("dev_in", []).append([dblock[c] for c in range(4)])
        assert all(a.shape[0] == LQ for a in pl["host_in"][0])
        self.pools[logn] = pl
        return pl

    def shape(self, logn: int, L: int):
        key = (logn, L)
        if key in self.shapes:
            return self.shapes[key]
        hefx = self.hefx
        qs = self.qprimes[:L]
        res = {
            "pQ": hefx.hefx_params_create(self.ctx, logn, qs),
            "pP": self.pparams(logn),
            "bc": hefx.hefx_bconv_plan_create(self.ctx, logn, qs, self.pprimes),
        }
        pl = self.pool(logn)
        res["mp"] = hefx.hefx_mult_plan_create(self.ctx, res["pQ"], res["pP"], res["bc"], pl["kQ"][0][:L],
                                               pl["kQ"][1][:L], pl["kP"][0], pl["kP"][1])
        self.shapes[key] = res
        return res

    def pparams(self, logn: int):
        if logn not in self.pparams_cache:
            self.pparams_cache[logn] = self.hefx.hefx_params_create(self.ctx, logn, self.pprimes)
        return self.pparams_cache[logn]

    def warm(self, logn: int, L: int) -> None:
        self.pool(logn)
        self.shape(logn, L)

    # ---------------------------------------------------------------- request lifecycle
    def _slot(self):
        """A free (device buffer, pinned output buffer, event) slot, sized for the largest
        request (N = 2^16, 36 limbs); slots are created on demand and reused."""
        if self.free_slots:
            return self.free_slots.pop()
        torch = self.torch
        n, L, K = 1 << 16, len(self.qprimes), N_SPECIAL
        return {"d": torch.empty((10 * L + 3 * K) * n, dtype=torch.int32, device="cuda"),
                "h": torch.empty((4 * L + 2 * K) * n, dtype=torch.int32, pin_memory=True),
                "ev": torch.cuda.Event()}

    def _resident_call(self, reqs, slots, s):
        """hefx_mult_front_batch over device-resident inputs; each slot's device buffer holds the
        request's outputs ([4L + 2K][N]) then its workspace ([2L + K][N])."""
        plans, ins, outs, works = [], [[], [], [], []], [], []
        for req, slot in zip(reqs, slots):
            res = self.shape(req.logn, req.L)
            pl = self.pool(req.logn)
            plans.append(res["mp"])
            for c, t in enumerate(pl["dev_in"][req.variant % self.variants]):
                ins[c].append(t)
            n = 1 << req.logn
            outs.append(slot["d"])
            works.append(slot["d"][(4 * req.L + 2 * N_SPECIAL) * n:])
        self.hefx.hefx_mult_front_batch(self.ctx, self.batch, plans, *ins, outs, works, s.cuda_stream)

    def launch(self, req: Request):
        """Enqueues one request as one hefx_mult_front_host call (one pitched upload of the four
        inputs, every stage, one read-back of the contiguous outputs) and a completion event
        (resident: one hefx_mult_front_batch call over its device-resident inputs)."""
        if self.resident:
            s = self.streams[self.next_stream]
            self.next_stream = (self.next_stream + 1) % len(self.streams)
            slot = self._slot()
            self._resident_call([req], [slot], s)
            slot["ev"].record(s)
            return {"ev": slot["ev"], "slot": slot, "stream": s}
        res = self.shape(req.logn, req.L)
        pl = self.pool(req.logn)
        s = self.streams[self.next_stream]
        self.next_stream = (self.next_stream + 1) % len(self.streams)
        slot = self._slot()
        a0, a1, b0, b1 = pl["host_in"][req.variant % self.variants]
        self.hefx.hefx_mult_front_host(self.ctx, res["mp"], a0, a1, b0, b1, slot["h"], slot["d"], s.cuda_stream)
        slot["ev"].record(s)
        return {"ev": slot["ev"], "slot": slot, "stream": s}

    def launch_group(self, reqs):
        """Enqueues requests of one ring degree as one batched native call and a completion
        event; returns one handle per request (sharing the event)."""
        s = self.streams[self.next_stream]
        self.next_stream = (self.next_stream + 1) % len(self.streams)
        if self.resident:
            slots = [self._slot() for _ in reqs]
            self._resident_call(reqs, slots, s)
            ev = slots[0]["ev"]
            ev.record(s)
            return [{"ev": ev, "slot": sl, "stream": s} for sl in slots]
        plans, ins, outs, bufs, slots = [], [[], [], [], []], [], [], []
        for req in reqs:
            res = self.shape(req.logn, req.L)
            pl = self.pool(req.logn)
            slot = self._slot()
            plans.append(res["mp"])
            for c, t in enumerate(pl["host_in"][req.variant % self.variants]):
                ins[c].append(t)
            outs.append(slot["h"])
            bufs.append(slot["d"])
            slots.append(slot)
        self.hefx.hefx_mult_front_batch_host(self.ctx, self.batch, plans, *ins, outs, bufs, s.cuda_stream)
        ev = slots[0]["ev"]
        ev.record(s)
        return [{"ev": ev, "slot": sl, "stream": s} for sl in slots]

    def retire(self, handle) -> None:
        """Returns a completed request's slot to the pool."""
        self.free_slots.append(handle["slot"])

    def done(self, handle) -> bool:
        return handle["ev"].query()

    def outputs(self, req: Request, handle):
        L, n = req.L, 1 << req.logn
        words = (4 * L + 2 * N_SPECIAL) * n
        src = handle["slot"]["d"][:words].cpu() if self.resident else handle["slot"]["h"][:words]
        o = src.numpy().view(np.uint32).reshape(-1, n)
        return (o[0:L].copy(), o[L:2 * L].copy(), np.concatenate([o[2 * L:3 * L], o[4 * L:4 * L + N_SPECIAL]]),
                np.concatenate([o[3 * L:4 * L], o[4 * L + N_SPECIAL:]]))

    def inputs_of(self, req: Request):
        """Host copies of the request's four input polynomials and its keys (for checks)."""
        pl = self.pool(req.logn)
        ins = [t[:req.L].numpy().view(np.uint32) for t in pl["host_in"][req.variant % self.variants]]
        keys = [np.concatenate([pl["kQ"][k][:req.L].cpu().numpy().view(np.uint32),
                                pl["kP"][k].cpu().numpy().view(np.uint32)]) for k in range(2)]
        return ins, keys

    def close(self):
        for res in self.shapes.values():
            self.hefx.hefx_mult_plan_destroy(res["mp"])
            self.hefx.hefx_bconv_plan_destroy(res["bc"])
            self.hefx.hefx_params_destroy(res["pQ"])
        for p in self.pparams_cache.values():
            self.hefx.hefx_params_destroy(p)
        if self.batch:
            self.hefx.hefx_mult_batch_destroy(self.batch)
            self.batch = None
        self.shapes, self.pparams_cache, self.pools = {}, {}, {}


def serve(requests, executor, budget_bytes: int = 40 << 30, max_slots: int | None = None,
          keep_outputs: bool = False):
    """Runs the requests (sorted by arrival) to completion in real time; returns stats.

    At most max_slots requests (default: 4 per executor stream) are in flight; later ones wait
    in the FIFO admission queue, so queueing shows up as latency instead of piling work onto
    the streams.  A stream completes its requests in order, so only the oldest request of
    each stream is polled."""
    requests = sorted(requests, key=lambda r: r.arrival)
    # the loop allocates many small objects; a cyclic-garbage pass over the whole process heap
    # in the middle of it stalls admission for tens of ms, so the collector waits until the end
    gc_was_enabled = gc.isenabled()
    gc.disable()
    try:
        return _serve(requests, executor, budget_bytes, max_slots, keep_outputs)
    finally:
        if gc_was_enabled:
            gc.enable()


def _serve(requests, executor, budget_bytes, max_slots, keep_outputs):
    nstreams = len(getattr(executor, "streams", [])) or 8
    adm = Admission(budget_bytes, max_slots if max_slots is not None else 4 * nstreams)
    fifo = collections.defaultdict(collections.deque)  # stream key -> in-flight (req, handle)
    t0 = time.perf_counter()
    i = 0
    max_active = 0
    host_launch = 0.0
    while i < len(requests) or adm.queue or adm.active:
        now = time.perf_counter() - t0
        while i < len(requests) and requests[i].arrival <= now:
            adm.submit(requests[i])
            i += 1
        admitted = list(adm.admit())
        if admitted and getattr(executor, "grouped", False):
            # continuous batching: requests admitted together run as groups of one ring degree
            by_n = collections.defaultdict(list)
            for req in admitted:
                by_n[req.logn].append(req)
            for group in by_n.values():
                for k in range(0, len(group), executor.max_group):
                    chunk = group[k:k + executor.max_group]
                    ta = time.perf_counter() - t0
                    for req in chunk:
                        req.admitted = ta
                    hs = executor.launch_group(chunk)
                    host_launch += time.perf_counter() - t0 - ta
                    for req, h in zip(chunk, hs):
                        fifo[id(h["stream"])].append((req, h))
        else:
            for req in admitted:
                req.admitted = time.perf_counter() - t0
                h = executor.launch(req)
                host_launch += time.perf_counter() - t0 - req.admitted
                fifo[id(h.get("stream")) if isinstance(h, dict) else 0].append((req, h))
        max_active = max(max_active, adm.active)
        for q in fifo.values():
            while q and executor.done(q[0][1]):
                req, h = q.popleft()
                req.completed = time.perf_counter() - t0
                req.status = "done"
                if keep_outputs:
                    req.outputs = executor.outputs(req, h)
                if hasattr(executor, "retire"):
                    executor.retire(h)
                adm.release(req)
        if not adm.active and not adm.queue and i < len(requests):
            wait = requests[i].arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.01))
    done = [r for r in requests if r.status == "done"]
    lat = np.array([r.completed - r.arrival for r in done]) if done else np.zeros(1)
    span = (max(r.completed for r in done) - min(r.arrival for r in done)) if done else 0.0
    return {
        "requests": len(requests), "completed": len(done),
        "rejected": sum(r.status == "rejected" for r in requests),
        "throughput_rps": len(done) / span if span > 0 else 0.0,
        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "max_active": max_active, "memory_high_water_bytes": adm.high_water,
        "host_launch_us_per_request": 1e6 * host_launch / max(1, sum(r.admitted >= 0 for r in requests)),
    }


def serve_native(requests, executor, budget_bytes: int = 40 << 30, max_slots: int | None = None,
                 keep_outputs: bool = False):
    """serve() with the request loop in native code (hefx_serve_run): the same admission,
    grouping and completion rules, for a resident grouped executor.  The result slots are the
    executor's (at most max_slots, default 4 per stream); with keep_outputs the results are
    read from their slots after the run (give at least as many slots as requests)."""
    assert executor.resident and executor.grouped, "the native loop serves resident, grouped requests"
    hefx, torch = executor.hefx, executor.torch
    requests = sorted(requests, key=lambda r: r.arrival)
    nslots = max_slots if max_slots is not None else 4 * len(executor.streams)
    slots = [executor._slot() for _ in range(nslots)]
    try:
        rows = []
        for req in requests:
            res = executor.shape(req.logn, req.L)
            a0, a1, b0, b1 = executor.pool(req.logn)["dev_in"][req.variant % executor.variants]
            rows.append((req.arrival, res["mp"], a0, a1, b0, b1, request_bytes(req.logn, req.L)))
        outs = [sl["d"] for sl in slots]
        # the workspace after the largest request's outputs ([4L + 2K][N] at L = 36, N = 2^16)
        works = [sl["d"][(4 * len(executor.qprimes) + 2 * N_SPECIAL) << 16:] for sl in slots]
        torch.cuda.synchronize()
        res_arr, stats = hefx.hefx_serve_run(executor.ctx, executor.batch, rows, executor.streams, outs, works,
                                             budget_bytes, executor.max_group)
        torch.cuda.synchronize()
        for k, req in enumerate(requests):
            r = res_arr[k]
            req.status = {hefx.SERVE_DONE: "done", hefx.SERVE_REJECTED: "rejected"}.get(r.status, "failed")
            req.admitted, req.completed = r.admitted_s, r.completed_s
            if keep_outputs and req.status == "done":
                req.outputs = executor.outputs(req, {"slot": slots[r.slot]})
    finally:
        executor.free_slots.extend(slots)
    done = [r for r in requests if r.status == "done"]
    lat = np.array([r.completed - r.arrival for r in done]) if done else np.zeros(1)
    span = (max(r.completed for r in done) - min(r.arrival for r in done)) if done else 0.0
    return {
        "requests": len(requests), "completed": len(done),
        "rejected": sum(r.status == "rejected" for r in requests),
        "throughput_rps": len(done) / span if span > 0 else 0.0,
        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "max_active": int(stats.max_active), "memory_high_water_bytes": int(stats.memory_high_water_bytes),
        "groups": int(stats.groups),
    }


def poisson_requests(seed: int, count: int, rate_hz: float, logn_choices=(13, 14, 15, 16), lmin=8, lmax=36,
                     variants: int = 2):
    """Seeded Poisson arrivals with N and L drawn uniformly per request."""
    t = inputs.poisson_arrivals(seed, count, rate_hz)
    r = inputs.splitmix64(inputs.derive_seed(seed, 7), 3 * count)
    out = []
    for k in range(count):
        logn = logn_choices[int(r[3 * k] % np.uint64(len(logn_choices)))]
        L = lmin + int(r[3 * k + 1] % np.uint64(lmax - lmin + 1))
        out.append(Request(k, logn, L, float(t[k]), variant=int(r[3 * k + 2] % np.uint64(variants))))
    return out
