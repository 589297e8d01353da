"""hefx benchmark: N = 2^16 limb-NTTs per second on one GB300.

Workload (one "step"): forward + inverse negacyclic NTT of a batch of 8 polynomials with
L = 24 RNS limbs of 28-bit primes, N = 2^16 (384 limb-NTTs), uniform synthetic residues.
Both hefx paths are timed (CUDA-core radix-2 under its two schedules, and the tensor-core
matrix NTT for each split and tile, when built); `value` is the fastest bit-exact
configuration, `paths` lists them all.  Inputs (48 MiB) are smaller than
L2, so a 256 MiB buffer is written between timed steps to flush it.

Contract: one JSON line on rank 0.  `python bench.py --impl reference` times the CPU oracle
instead (the reference arm of this workload).  Under torchrun every rank runs an
independent replica (the method has no exchange step), timed between barriers.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LOGN, L, BATCH = 16, 24, 8
N = 1 << LOGN
UNITS_PER_STEP = 2 * BATCH * L             # limb-NTTs per step (forward + inverse)
BYTES_PER_UNIT = 2 * N * 4                 # one read and one write of a limb per transform
METRIC = "N=2^16 limb-NTTs/s, int8-tensor-core vs CUDA-core path, bit-exact; % roofline"
WORKLOAD = "CKKS-shaped NTT: N=2^16, L=24 28-bit limbs, batch 8, forward+inverse"
L2_FLUSH_BYTES = 256 << 20


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), float(p.get("bf16_tflops_sustained", 0)), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


# ----------------------------------------------------------------------------- clocks

class NvmlSampler:
    """Samples SM clocks and throttle reasons every 0.5 ms through NVML (ctypes, read-only
    queries) while the timed region runs; the GPU is found by its PCI bus id."""

    # clock-event reason bits (nvml.h)
    REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, device: int):
        import ctypes
        self.ct = ctypes
        self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
        if self.nvml.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        import torch
        pr = torch.cuda.get_device_properties(device)
        bus = f"{getattr(pr, 'pci_domain_id', 0):08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0".encode()
        if self.nvml.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(self.h)) != 0:
            raise RuntimeError("GPU not found by PCI bus id")
        self.reason_fn = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nvml.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        self.max_mhz = float(mx.value) if self.nvml.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0 else None
        self.samples, self.reasons, self.stop = [], set(), threading.Event()

    def _poll(self):
        ct = self.ct
        clk, rs = ct.c_uint(), ct.c_ulonglong()
        while not self.stop.is_set():
            if self.nvml.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(clk)) == 0:  # NVML_CLOCK_SM
                self.samples.append(float(clk.value))
            if self.reason_fn(self.h, ct.byref(rs)) == 0:
                self.reasons.update(k for k, bit in self.REASONS.items() if rs.value & bit)
            time.sleep(0.0005)

    def __enter__(self):
        self.thread = threading.Thread(target=self._poll, daemon=True)
        self.thread.start()
        return self

    def __exit__(self, *exc):
        self.stop.set()
        self.thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples), "source": "nvml"}


def clock_sampler(device: int):
    """NVML sampler where the driver's library loads, else nvidia-smi polling."""
    try:
        return NvmlSampler(device)
    except Exception:
        return ClockSampler(device)


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle

def _oracle_worker(args):
    kind, seed, budget_s, primes = args
    import oracle as orc
    from paper_2501_07047_gb300 import inputs
    done = 0
    t0 = time.perf_counter()
    i = 0
    while time.perf_counter() - t0 < budget_s:
        if kind == "ntt":  # forward + inverse limb-NTT pair
            q = primes[i % len(primes)]
            a = inputs.uniform_residues(inputs.derive_seed(seed, i), N, q)
            orc.intt(orc.ntt(a, q), q)
            done += 2
        elif kind == "polymul":  # one N = 2^16 limb product (NTT, Hadamard, INTT)
            q = primes[i % len(primes)]
            a = inputs.uniform_residues(inputs.derive_seed(seed, i, 0), N, q)
            b = inputs.uniform_residues(inputs.derive_seed(seed, i, 1), N, q)
            orc.polymul(a, b, q)
            done += 1
        else:  # basis conversion of 2^12 coefficients, 24 -> 8 limbs (config 3's shape)
            qs, ps = primes[:24], inputs.special_primes(8)
            x = inputs.residue_tensor(inputs.derive_seed(seed, i), 1, qs, 4096)[0]
            orc.bconv(x, qs, ps)
            done += 4096
        i += 1
    return done, time.perf_counter() - t0


def time_oracle(budget_s: float, cores: int | None = None, kind: str = "ntt"):
    """Runs the oracle on every host core (spawned processes, one per core) for a bounded time
    and returns the throughput over all cores: forward + inverse N = 2^16 limb-NTTs (kind
    "ntt", the headline unit), N = 2^16 limb products ("polymul") or 24 -> 8 basis-conversion
    coefficients ("bconv")."""
    import oracle as orc
    orc.build()
    from paper_2501_07047_gb300 import inputs
    primes = inputs.source_primes(L)
    cores = cores or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(kind, 1000 + w, budget_s, primes) for w in range(cores)])
    wall = time.perf_counter() - t0
    units = sum(r[0] for r in res)
    longest = max(r[1] for r in res)
    unit, what = {"ntt": ("limb-NTT/s", "N=2^16 limb-NTTs (forward+inverse pairs over the 24 limb primes)"),
                  "polymul": ("limb-products/s", "N=2^16 limb products (NTT, Hadamard, INTT)"),
                  "bconv": ("coeffs/s", "basis-conversion coefficients (24 -> 8 limbs)")}[kind]
    return {"value": units / longest, "unit": unit, "cores": cores, "kind": "oracle",
            "sample": f"{units} {what} in {longest:.1f} s per core, {cores} processes, wall {wall:.1f} s"}


def cpu_baseline_extra(budget_s: float):
    """The oracle's other units (SURVEY 8(d) CPU plan): one-thread limb-NTT/s, and limb
    products and basis-conversion coefficients per second on every core."""
    return {"ntt_1_thread": time_oracle(budget_s, cores=1, kind="ntt"),
            "polymul_all_cores": time_oracle(budget_s, kind="polymul"),
            "bconv_all_cores": time_oracle(budget_s, kind="bconv")}


# ----------------------------------------------------------------------------- GPU arm

def max_over_ranks(ms: float, dist=None, device: str = "cpu") -> float:
    """The slowest rank's time (every rank gets it); the time itself without a process group."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, units_per_step: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_step * steps / (total_ms / 1e3)


def run_gpu(args):
    import torch
    from paper_2501_07047_gb300 import build, hefx, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # start the CPU-baseline pool (spawn) before the first CUDA call
    cpu_baseline = cpu_extra = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_baseline = time_oracle(args.cpu_seconds)
        cpu_extra = cpu_baseline_extra(max(1.0, args.cpu_seconds / 4))

    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    ctx = hefx.hefx_create(local)
    primes = inputs.source_primes(L)
    params = hefx.hefx_params_create(ctx, LOGN, primes)
    host = inputs.residue_tensor(inputs.derive_seed(2, rank), BATCH, primes, N)
    host_t = torch.from_numpy(host.view(np.int32).copy())
    data0 = host_t.cuda()
    data = data0.clone()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def available(path):
        st = hefx.raw_status("hefx_ntt_fwd", ctx, params, data.data_ptr(), 0, hefx.PATHS[path], stream.cuda_stream)
        return st == hefx.HEFX_OK

    # timed configurations: the CUDA-core path under both of its schedules (one launch of 8-CTA
    # clusters; two launches, column pass then block pass) and the tensor path with each split
    # and GEMM tile width
    configs = [("cudacore", "cudacore", 0, (0, 0), "auto"), ("cudacore_2p", "cudacore", 0, (0, 0), "two_pass")]
    if available("tensor"):
        # two-factor 256 x 256 and the three-factor 64 x 32 x 32 split, each with both tiles
        configs += [("tensor", "tensor", 64, (0, 0), "auto"), ("tensor_t32", "tensor", 32, (0, 0), "auto"),
                    ("tensor_3f", "tensor", 64, (6, 5), "auto"), ("tensor_3f_t32", "tensor", 32, (6, 5), "auto")]
    # Whole-job throughput: the K steps are independent batches, and a stream of them runs
    # with steps k and k + 1 overlapping on PIPE_STREAMS streams, so that the GPU is not idle
    # in each transform's last, partial wave of clusters (192 rows over 89 co-resident
    # clusters leave about a fifth of a launch nearly empty).  PIPE_BATCHES rotating input
    # batches of 48 MiB (192 MiB) exceed L2, so these steps need no flush.  One parameter set
    # per stream: the tensor path's digit workspace lives in the parameter set.  The
    # per-launch times (fwd_ms / inv_ms, the roofline) come from the serialized loop below.
    PIPE_STREAMS, PIPE_BATCHES = 2, 4
    pipe_params = [hefx.hefx_params_create(ctx, LOGN, primes) for _ in range(PIPE_STREAMS)]
    pipe_bufs = [data0.clone() for _ in range(PIPE_BATCHES)]
    pipe_streams = [torch.cuda.Stream() for _ in range(PIPE_STREAMS)]

    def pipelined(path, tile, split, sched):
        for pp in pipe_params:
            hefx.hefx_params_set_cc_schedule(ctx, pp, sched)
            if tile:
                hefx.hefx_params_set_tensor_config(ctx, pp, split[0], tile, split[1])

        def step(k):
            s, pp, b = pipe_streams[k % PIPE_STREAMS], pipe_params[k % PIPE_STREAMS], pipe_bufs[k % PIPE_BATCHES]
            hefx.hefx_ntt_fwd(ctx, pp, b, BATCH, path, s)
            hefx.hefx_ntt_inv(ctx, pp, b, BATCH, path, s)

        for s in pipe_streams:
            s.wait_stream(stream)
        for k in range(max(args.warmup, 1) * PIPE_BATCHES):
            step(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e1.record(stream)
        joins = [torch.cuda.Event() for _ in pipe_streams]
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        with clock_sampler(local) as clk:
            for _ in range(4):
                flush.fill_(-1)  # device work queued ahead of the timed launches (outside the events)
            e0.record(stream)
            for s in pipe_streams:
                s.wait_stream(stream)
            for k in range(args.steps):
                step(k)
            for s, j in zip(pipe_streams, joins):
                j.record(s)
                stream.wait_event(j)
            e1.record(stream)
            torch.cuda.synchronize()
        if dist:
            dist.barrier()
        for b in pipe_bufs:  # every batch made whole round trips
            assert torch.equal(b, data0), f"{path}: pipelined round trip mismatch"
        return max_over_ranks(e0.elapsed_time(e1), dist, "cuda"), clk.summary()

    results = {}
    for name, path, tile, split, sched in configs:
        hefx.hefx_params_set_cc_schedule(ctx, params, sched)
        if tile:
            hefx.hefx_params_set_tensor_config(ctx, params, split[0], tile, split[1])
        # correctness gate: INTT(NTT(x)) == x on the bench data before timing
        data.copy_(data0)
        hefx.hefx_ntt_fwd(ctx, params, data, BATCH, path, stream)
        hefx.hefx_ntt_inv(ctx, params, data, BATCH, path, stream)
        torch.cuda.synchronize()
        assert torch.equal(data, data0), f"{path}: round trip mismatch"
        for _ in range(args.warmup):
            hefx.hefx_ntt_fwd(ctx, params, data, BATCH, path, stream)
            hefx.hefx_ntt_inv(ctx, params, data, BATCH, path, stream)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
        for e in (x for row in ev for x in row):  # torch creates an event at its first record:
            e.record(stream)                      # do that here, not between a step's launches
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        with clock_sampler(local) as clk:
            t_wall = time.perf_counter()
            # queue some GPU work first, so that the host's launches run ahead of the device
            # from the first timed step on (outside the events)
            for _ in range(4):
                flush.fill_(-1)
            for k in range(args.steps):
                flush.fill_(k)  # write 256 MiB > L2 between timed steps (outside the events)
                ev[k][0].record(stream)
                hefx.hefx_ntt_fwd(ctx, params, data, BATCH, path, stream)
                ev[k][1].record(stream)
                hefx.hefx_ntt_inv(ctx, params, data, BATCH, path, stream)
                ev[k][2].record(stream)
            torch.cuda.synchronize()
            t_wall = time.perf_counter() - t_wall
        if dist:
            dist.barrier()
        fwd_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
        inv_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
        step_ms = sum(fwd_ms) / args.steps + sum(inv_ms) / args.steps
        total_ms = step_ms * args.steps
        total_ms = max_over_ranks(total_ms, dist, "cuda")
        results[name] = {
            "path": path, "tile": tile, "split": split, "schedule": sched,
            "ms_per_step": total_ms / args.steps,
            "value": job_value(world, UNITS_PER_STEP, args.steps, total_ms),
            "fwd_ms": statistics.mean(fwd_ms), "inv_ms": statistics.mean(inv_ms),
            "wall_s": t_wall, "clocks": clk.summary(),
            "launches_per_step": (4 if sched == "two_pass" else 2) if path == "cudacore" else (6 if not split[1] else 8),
        }
        pipe_ms, pipe_clk = pipelined(path, tile, split, sched)
        results[name].update({"ms_per_step_pipelined": pipe_ms / args.steps,
                              "value_pipelined": job_value(world, UNITS_PER_STEP, args.steps, pipe_ms),
                              "clocks_pipelined": pipe_clk})

    if available("tensor"):
        hefx.hefx_params_set_tensor_config(ctx, params, 0, 64, 0)
    # the headline is the library's own choice for this shape (AUTO: the cluster schedule at 192
    # rows) or a tensor configuration; the explicit two-pass schedule is listed for comparison
    best_name = max((k for k in results if k != "cudacore_2p"), key=lambda p: results[p]["value_pipelined"])
    r = results[best_name]
    best = r["path"]
    hefx.hefx_params_set_cc_schedule(ctx, params, r["schedule"])
    if best == "tensor":
        hefx.hefx_params_set_tensor_config(ctx, params, r["split"][0], r["tile"], r["split"][1])

    # end to end through the public calls with host buffers: per step the pinned H2D of the
    # batch, fwd, inv and the D2H of the result, over three streams and three device buffers
    # (hostio.NttRoundTrip) so that step k+1's upload and step k-1's download run under step
    # k's transforms (measured: whole-batch chunks 0.314 ms/step, per-polynomial chunks 0.486:
    # 24-row launches underfill the GPU; the copies alone take 0.308 ms at 327 GB/s both ways)
    from paper_2501_07047_gb300.hostio import NttRoundTrip
    pinned_in = host_t.pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    rt = NttRoundTrip(ctx, params, L, N, chunk=BATCH, path=best)
    for _ in range(2):
        rt.run(pinned_in, pinned_out)
    rt.join()
    torch.cuda.synchronize()
    assert torch.equal(pinned_out, host_t)
    pinned_out.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        rt.run(pinned_in, pinned_out)
    rt.join(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    assert torch.equal(pinned_out, host_t)

    hbm, bf16, bf16_s, src = peaks()
    units_per_launch = BATCH * L

    def roof_cudacore(rr):
        dom = max(rr["fwd_ms"], rr["inv_ms"])
        achieved = units_per_launch * BYTES_PER_UNIT / (dom / 1e3) / 1e9
        which = "fwd" if rr["fwd_ms"] >= rr["inv_ms"] else "inv"
        cluster = rr["schedule"] != "two_pass"  # AUTO runs the cluster kernel at 192 rows
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": profile_traffic("ntt_cc", which) if cluster else None,
                "kernel": ("ntt_cc_kernel<16, " + which.upper() + ">") if cluster else
                          ("two-pass " + which + " transform (column and block kernels, timed together)"),
                "algorithmic_bytes_per_launch": units_per_launch * BYTES_PER_UNIT,
                "peak_source": f"{src} hbm_gbs"}

    def roof_tensor(rr):
        # one transform = digitize + two (three) digit-GEMM launches; flops are the GEMMs' digit MACs
        dom = max(rr["fwd_ms"], rr["inv_ms"])
        flops = tensor_flops_per_limb_ntt(*rr["split"]) * units_per_launch
        achieved = flops / (dom / 1e3) / 1e12
        return {"bound": "tensor", "achieved": round(achieved, 1), "peak": bf16, "unit": "TFLOP/s",
                "frac": round(achieved / bf16, 4), "traffic": None,
                "kernel": "tensor-path " + ("forward" if rr["fwd_ms"] >= rr["inv_ms"] else "inverse")
                          + " transform (digitize + 2 bat digit-GEMM launches, timed together)",
                "algorithmic_flops_per_transform": flops,
                "peak_source": f"{src} bf16_tflops (fp16 dense runs at the bf16 rate)"}

    roof = roof_cudacore(r) if best == "cudacore" else roof_tensor(r)
    roof_other = None
    tensor_names = [k for k in results if results[k]["path"] == "tensor"]
    if tensor_names and best != "tensor":
        roof_other = roof_tensor(results[max(tensor_names, key=lambda k: results[k]["value"])])
    roof_tensor_configs = {k: {"tile_outputs": results[k]["tile"],
                               "split": "x".join(str(f) for f in tensor_split(*results[k]["split"])),
                               "frac": roof_tensor(results[k])["frac"],
                               "achieved_TFLOP_s": roof_tensor(results[k])["achieved"]} for k in tensor_names}

    line = {
        "metric": METRIC, "value": round(r["value_pipelined"], 1), "unit": "limb-NTT/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r["ms_per_step_pipelined"], 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "limbs": L, "batch": BATCH, "path": best,
                   "units_per_step": UNITS_PER_STEP,
                   "timing": f"value: the K steps as independent batches, step k on stream k mod {PIPE_STREAMS} "
                             f"(neighbouring steps overlap); per-launch times and the roofline: serialized steps",
                   "l2": f"value: inputs larger than L2 ({PIPE_BATCHES} rotating batches, "
                         f"{PIPE_BATCHES * BATCH * L * N * 4 >> 20} MiB); serialized steps: flushed (256 MiB write) between steps",
                   "parallelism": f"replicas x{world}"},
        "value_serialized": round(r["value"], 1), "ms_per_step_serialized": round(r["ms_per_step"], 5),
        "paths": {p: {"value": round(v["value_pipelined"], 1), "ms_per_step": round(v["ms_per_step_pipelined"], 5),
                      "value_serialized": round(v["value"], 1), "ms_per_step_serialized": round(v["ms_per_step"], 5),
                      "fwd_ms": round(v["fwd_ms"], 5), "inv_ms": round(v["inv_ms"], 5)} for p, v in results.items()},
        "config_choice": best_name,
        "roofline": roof,
        # the same bytes over the whole pipelined job: every launch's algorithmic bytes over the
        # device time of the K overlapping steps (what the GPU sustained, tails included)
        "roofline_job": ({"bound": "hbm", "unit": "GB/s", "peak": hbm,
                          "achieved": round(2 * units_per_launch * BYTES_PER_UNIT / (r["ms_per_step_pipelined"] / 1e3) / 1e9, 1),
                          "frac": round(2 * units_per_launch * BYTES_PER_UNIT / (r["ms_per_step_pipelined"] / 1e3) / 1e9 / hbm, 4),
                          "basis": "2 launches x algorithmic bytes per step / pipelined device time per step"}
                         if best == "cudacore" else None),
        "roofline_tensor_path": roof_other,
        "roofline_tensor_configs": roof_tensor_configs,
        "clocks": r["clocks_pipelined"],
        "clocks_serialized": r["clocks"],
        "e2e": {"value": round(job_value(world, UNITS_PER_STEP, args.steps, e2e_ms), 1), "unit": "limb-NTT/s",
                "h2d_bytes_per_step": int(host.nbytes), "d2h_bytes_per_step": int(host.nbytes),
                "overlap": "3 streams, 3 device buffers: step k+1 H2D and step k-1 D2H under step k's transforms"},
        "gpu_launches": r["launches_per_step"] * args.steps,
    }
    if cpu_baseline:
        line["cpu_baseline"] = cpu_baseline
        line["cpu_baseline_other_units"] = cpu_extra
    hefx.hefx_params_destroy(params)
    for pp in pipe_params:
        hefx.hefx_params_destroy(pp)
    del data, data0, flush, pipe_bufs
    torch.cuda.empty_cache()
    if not args.no_extras and world == 1:
        runs = {"bconv_config3": bench_bconv, "batch_config4": bench_batch, "he_mult": bench_he_mult,
                "reduction_ablation": bench_reduction_ablation, "paper_ntt_table": bench_paper_ntt_table}
        chosen = [k for k in runs if args.extras is None or k in args.extras.split(",")]
        line["extra"] = {k: runs[k](ctx, args) for k in chosen}
        if not args.no_serve and (args.extras is None or "serving_config5" in args.extras.split(",")):
            line["extra"]["serving_config5"] = bench_serving(ctx, args)
    hefx.hefx_destroy(ctx)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def _events_time(fn, steps, flush, stream):
    import torch
    ms = []
    for k in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)  # created at the first record: before the flush, not inside the timed span
        e1.record(stream)
        flush.fill_(k)  # also the device work the host's launch in fn() runs ahead of
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def _pipelined_time(fn, bufs, calls, stream):
    """Milliseconds per call of `calls` calls fn(buf, stream_i), call k on stream k mod 2 with
    buffer k mod len(bufs), neighbouring calls overlapping (device time, CUDA events)."""
    import torch
    sts = [torch.cuda.Stream() for _ in range(2)]
    for k in range(4):
        fn(bufs[k % len(bufs)], sts[k % 2])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    for st in sts:
        st.wait_stream(stream)
    e0.record(stream)
    for st in sts:
        st.wait_stream(stream)
    for k in range(calls):
        fn(bufs[k % len(bufs)], sts[k % 2])
    for st in sts:
        stream.wait_stream(st)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / calls


def bench_bconv(ctx, args):
    """RNS basis conversion 16 x 24 limbs x 2^16 -> 8 limbs, both paths."""
    import torch
    from paper_2501_07047_gb300 import hefx, inputs
    B, Lq, Lp, logn = 16, 24, 8, 16
    n = 1 << logn
    qs, ps = inputs.source_primes(Lq), inputs.special_primes(Lp)
    plan = hefx.hefx_bconv_plan_create(ctx, logn, qs, ps)
    x = inputs.residue_tensor(inputs.derive_seed(3, 0), B, qs, n)
    dx = torch.from_numpy(x.view(np.int32).copy()).cuda()
    dy = torch.empty((B, Lp, n), dtype=torch.int32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    hbm, _, _, src = peaks()
    out = {"workload": "BConv 16 x 24 limbs (28-bit) x 2^16 -> 8 limbs (30-bit)", "bytes_per_call": (Lq + Lp) * 4 * n * B}
    ref = None
    for path in ("cudacore", "tensor"):
        hefx.hefx_basis_convert(ctx, plan, dx, dy, B, path, s)
        torch.cuda.synchronize()
        if ref is None:
            ref = dy.clone()
        assert torch.equal(dy, ref), "paths disagree"
        for _ in range(3):
            hefx.hefx_basis_convert(ctx, plan, dx, dy, B, path, s)
        ms = _events_time(lambda: hefx.hefx_basis_convert(ctx, plan, dx, dy, B, path, s), args.steps, flush, s)
        gbs = out["bytes_per_call"] / (ms / 1e3) / 1e9
        out[path] = {"ms": round(ms, 5), "coeffs_per_s": round(B * n / (ms / 1e3), 1), "GB_s": round(gbs, 1),
                     "hbm_frac": round(gbs / hbm, 4)}
    out["peak"] = f"{hbm} GB/s ({src} hbm_gbs)"
    hefx.hefx_bconv_plan_destroy(plan)
    del dx, dy
    # the paper's skewed conversion shapes (N = 2^16, one polynomial and a batch of 8), both paths
    shapes = {}
    for Lq2, Lp2 in ((12, 28), (12, 36), (16, 40), (24, 56)):
        qs2, ps2 = inputs.source_primes(Lq2), inputs.special_primes(Lp2)
        plan2 = hefx.hefx_bconv_plan_create(ctx, logn, qs2, ps2)
        row = {}
        for B2 in (1, 8):
            x2 = inputs.residue_tensor(inputs.derive_seed(3, Lq2, Lp2), B2, qs2, n)
            dx2 = torch.from_numpy(x2.view(np.int32).copy()).cuda()
            dy2 = torch.empty((B2, Lp2, n), dtype=torch.int32, device="cuda")
            ref2 = None
            for path in ("cudacore", "tensor"):
                st = hefx.raw_status("hefx_basis_convert", ctx, plan2, dx2.data_ptr(), dy2.data_ptr(), 0,
                                     hefx.PATHS[path], s.cuda_stream)
                if st != hefx.HEFX_OK:
                    row[f"{path}_b{B2}_us"] = None
                    continue
                hefx.hefx_basis_convert(ctx, plan2, dx2, dy2, B2, path, s)
                torch.cuda.synchronize()
                if ref2 is None:
                    ref2 = dy2.clone()
                assert torch.equal(dy2, ref2), "paths disagree"
                for _ in range(3):
                    hefx.hefx_basis_convert(ctx, plan2, dx2, dy2, B2, path, s)
                ms = _events_time(lambda: hefx.hefx_basis_convert(ctx, plan2, dx2, dy2, B2, path, s),
                                  max(5, args.steps // 2), flush, s)
                row[f"{path}_b{B2}_us"] = round(ms * 1e3, 2)
        shapes[f"{Lq2}->{Lp2}"] = row
        hefx.hefx_bconv_plan_destroy(plan2)
    out["paper_shapes_n65536"] = shapes
    out["paper_context_us"] = "TPU v6e one tensor core, BAT: 12->28 135.91, 12->36 147.28, 16->40 65.77, 24->56 94.67"
    return out


def bench_paper_ntt_table(ctx, args):
    """The shapes of the paper's NTT-throughput table (Sec. V-B): Sets A / B / C, N = 2^12 /
    2^13 / 2^14 with L = 4 / 8 / 15 limbs of 28-bit primes, forward NTTs of a batch of
    polynomials (the paper's batches for one TPU v6e tensor core, 32 / 16 / 16, and batches that
    fill the GPU), every path that is built; thousands of polynomial NTTs (all L limbs) and of
    limb-NTTs per second."""
    import torch
    from paper_2501_07047_gb300 import hefx, inputs
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    out = {"paper_context_KNTT_s": {"A": {"TPU v6e-8": 14668, "TPU v4-4": 1284, "WarpDrive A100": 12181},
                                    "B": {"TPU v6e-8": 3850, "TPU v4-4": 323, "WarpDrive A100": 4675},
                                    "C": {"TPU v6e-8": 793, "TPU v4-4": 75, "WarpDrive A100": 2088}}}
    for name, logn, Lset, pbatch in (("A", 12, 4, 32), ("B", 13, 8, 16), ("C", 14, 15, 16)):
        primes = inputs.source_primes(Lset)
        params = hefx.hefx_params_create(ctx, logn, primes)
        res = {"N": 1 << logn, "L": Lset}
        for batch in (pbatch, 16 * pbatch, 64 * pbatch):
            host = inputs.residue_tensor(inputs.derive_seed(6, logn, batch), batch, primes, 1 << logn)
            d0 = torch.from_numpy(host.view(np.int32).copy()).cuda()
            for path in ("cudacore", "tensor"):
                d = d0.clone()
                if hefx.raw_status("hefx_ntt_fwd", ctx, params, d.data_ptr(), 0, hefx.PATHS[path], s.cuda_stream) != 0:
                    continue
                hefx.hefx_ntt_fwd(ctx, params, d, batch, path, s)
                hefx.hefx_ntt_inv(ctx, params, d, batch, path, s)
                torch.cuda.synchronize()
                assert torch.equal(d, d0), f"paper table {name} {path}: round trip mismatch"
                ms = _events_time(lambda: hefx.hefx_ntt_fwd(ctx, params, d, batch, path, s), 20, flush, s)
                res[f"{path}_batch{batch}"] = {"us": round(ms * 1e3, 2),
                                               "KNTT_s_polys": round(batch / (ms / 1e3) / 1e3, 1),
                                               "K_limb_NTT_s": round(batch * Lset / (ms / 1e3) / 1e3, 1)}
                if path == "cudacore" and batch == 64 * pbatch:
                    # a stream of such calls: two streams, two batches of at least 128 MiB (more
                    # than L2 together), neighbouring calls overlapping
                    pm = _pipelined_time(lambda b, st: hefx.hefx_ntt_fwd(ctx, params, b, batch, path, st),
                                         [d, d0.clone()], 20, s)
                    res[f"{path}_batch{batch}_stream"] = {"us_per_call": round(pm * 1e3, 2),
                                                          "KNTT_s_polys": round(batch / (pm / 1e3) / 1e3, 1)}
        hefx.hefx_params_destroy(params)
        out[name] = res
    return out


def bench_reduction_ablation(ctx, args):
    """The paper's modular-reduction ablation (Sec. V-F) on GB300: Shoup / Montgomery / Barrett
    twiddle products in the CUDA-core NTT (N = 2^16, L = 24, batch 1 and 8, fwd + inv) and
    Montgomery / Barrett VecModMul over the same data.  Results are identical across variants."""
    import torch
    from paper_2501_07047_gb300 import hefx, inputs
    primes = inputs.source_primes(L)
    params = hefx.hefx_params_create(ctx, LOGN, primes)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    host = inputs.residue_tensor(inputs.derive_seed(2, 99), BATCH, primes, N)
    d0 = torch.from_numpy(host.view(np.int32).copy()).cuda()
    d = d0.clone()
    out = {"workload": "N=2^16, L=24 28-bit limbs; NTT = fwd + inv per batch; VecModMul over batch 8",
           "ntt_limb_ntt_per_s": {}, "vec_mod_mul_GB_s": {}}
    ref = None
    steps = max(5, args.steps // 2)
    for red in ("shoup", "montgomery", "barrett"):
        hefx.hefx_params_set_reduction(ctx, params, red, "montgomery")
        d.copy_(d0)
        hefx.hefx_ntt_fwd(ctx, params, d, BATCH, "cudacore", s)
        torch.cuda.synchronize()
        if ref is None:
            ref = d.clone()
        assert torch.equal(d, ref), f"{red}: forward NTT differs"
        for b in (1, BATCH):
            def step():
                hefx.hefx_ntt_fwd(ctx, params, d, b, "cudacore", s)
                hefx.hefx_ntt_inv(ctx, params, d, b, "cudacore", s)
            for _ in range(3):
                step()
            ms = _events_time(step, steps, flush, s)
            out["ntt_limb_ntt_per_s"][f"{red}_batch{b}"] = round(2 * b * L / (ms / 1e3), 1)
    hefx.hefx_params_set_reduction(ctx, params, "shoup", "montgomery")
    y = d0.clone()
    z = torch.empty_like(d0)
    zref = None
    for red in ("montgomery", "barrett", "bat_lazy"):  # bat_lazy: tensor-core MMA of the high bytes
        hefx.hefx_params_set_reduction(ctx, params, "shoup", red)
        hefx.hefx_vec_mod_mul(ctx, params, d0, y, z, BATCH, s)
        torch.cuda.synchronize()
        if zref is None:
            zref = z.clone()
        assert torch.equal(z, zref), f"{red}: VecModMul differs"
        ms = _events_time(lambda: hefx.hefx_vec_mod_mul(ctx, params, d0, y, z, BATCH, s), steps, flush, s)
        out["vec_mod_mul_GB_s"][red] = round(3 * 4 * BATCH * L * N / (ms / 1e3) / 1e9, 1)
    hefx.hefx_params_destroy(params)
    return out


def bench_he_mult(ctx, args):
    """HE-Mult (tensor product + dnum-digit hybrid key switching) and Rescale of one ciphertext
    pair at N = 2^16, the shapes of the paper's HE-operator table (L, log q, dnum) = (48, 28, 3)
    and (24, 28, 3); K = alpha = L / dnum special 30-bit primes.  Synthetic keys and inputs."""
    import torch
    from paper_2501_07047_gb300 import inputs
    from paper_2501_07047_gb300.hemult import HeMult
    logn, n = 16, 1 << 16
    res = {"workload": "HE-Mult = tensor product + relinearisation (ModUp, key inner product, ModDown); "
                       "Rescale = INTT, rescale, NTT; one ciphertext pair, N = 2^16",
           "paper_context_us": "CROSS TPU v6e-8 (48, 28, 3): HE-Mult 487, Rescale 74 (Table of HE operators)"}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    for L, dnum in ((48, 3), (24, 3)):
        alpha = -(-L // dnum)
        qs, ps = inputs.source_primes(L), inputs.special_primes(alpha)
        hm = HeMult(ctx, logn, qs, ps, alpha)
        qp = list(qs) + list(ps)

        def d(a):
            return torch.from_numpy(np.ascontiguousarray(a).view(np.int32).copy()).cuda()

        ins = [d(inputs.residue_tensor(inputs.derive_seed(6, L, c), 1, qs, n)[0]) for c in range(4)]
        evk = d(np.stack([np.stack([inputs.residue_tensor(inputs.derive_seed(6, L, 10 + j, k), 1, qp, n)[0]
                                    for k in range(2)]) for j in range(hm.dnum)]))
        cq = torch.empty((2, L, n), dtype=torch.int32, device="cuda")
        out = torch.empty((2, L - 1, n), dtype=torch.int32, device="cuda")
        for _ in range(3):
            hm.run(*ins, evk, cq, s, rescale=False)
            hm.rescale(cq.clone(), out, s)
        steps = max(5, args.steps // 2)
        mult_ms = _events_time(lambda: hm.run(*ins, evk, cq, s, rescale=False), steps, flush, s)
        cw = cq.clone()
        resc_ms = _events_time(lambda: hm.rescale(cw, out, s), steps, flush, s)
        # the same sequence replayed as one CUDA graph (no per-call host submission)
        g = hm.capture(*ins, evk, cq, rescale=False)
        ref = cq.clone()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(cq, ref), "graph replay differs from the eager run"
        graph_ms = _events_time(g.replay, steps, flush, s)
        res[f"L{L}_dnum{dnum}"] = {"he_mult_us": round(mult_ms * 1e3, 1), "he_mult_graph_us": round(graph_ms * 1e3, 1),
                                   "rescale_us": round(resc_ms * 1e3, 1), "K": alpha,
                                   "launches_he_mult": hm.launches(rescale=False),
                                   "launches_rescale": hm.launches(rescale=True) - hm.launches(rescale=False)}
        del g
        hm.close()
        del ins, evk, cq, out, cw
    return res


def bench_batch(ctx, args):
    """256 uneven polynomial-product jobs, one graph launch per batch."""
    import torch
    from paper_2501_07047_gb300 import hefx, inputs
    from paper_2501_07047_gb300.batch import UnevenBatch
    shapes = inputs.uneven_jobs(inputs.derive_seed(4), 256)
    batch = UnevenBatch(ctx, shapes, seed=4, fill=False)
    try:
        s = torch.cuda.Stream()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
        with torch.cuda.stream(s):
            for _ in range(3):
                batch.run(s)
            ms = _events_time(lambda: batch.run(s), max(5, args.steps // 4), flush, s)
        cl = batch.coeff_limbs()
        return {"workload": "256 jobs, N in {2^12..2^16}, L in [4, 32]; NTT(a), INTT(NTT(b) o NTT(a))",
                "ms_per_batch": round(ms, 4), "jobs_per_s": round(256 / (ms / 1e3), 1),
                "coeff_limbs_per_s": round(cl / (ms / 1e3), 1), "coeff_limbs": cl,
                "hbm_bytes_per_batch": 20 * cl, "GB_s": round(20 * cl / (ms / 1e3) / 1e9, 1),
                "launches_per_batch": hefx.hefx_batch_plan_launches(batch.plan), "graph": True}
    finally:
        batch.close()


def bench_serving(ctx, args):
    """Poisson arrival-rate sweep of ciphertext-multiply requests, 40 GB admission budget:
    continuous batching (requests admitted together run as groups of one ring degree in shared
    launches) and, for comparison at the top rates, one native call per request."""
    import torch
    from paper_2501_07047_gb300.serve import N_SPECIAL, GpuExecutor, poisson_requests, serve, serve_native
    res = {"workload": "HE-Mult front half, N in {2^13..2^16}, L in [8, 36], 8 special primes", "budget_GB": 40}
    # the ceiling the host link sets: every request uploads 4 L N words and reads back
    # (4 L + 2 K) N words; the link rate is measured here with both directions at once
    mix = poisson_requests(inputs_seed(5, 0), 2000, 1.0)
    bytes_req = statistics.mean(4 * ((4 * r.L) + (4 * r.L + 2 * N_SPECIAL)) * (1 << r.logn) for r in mix)
    nb = 256 << 20
    h_up = torch.empty(nb // 4, dtype=torch.int32).pin_memory()
    h_dn = torch.empty(nb // 4, dtype=torch.int32).pin_memory()
    d_up = torch.empty(nb // 4, dtype=torch.int32, device="cuda")
    d_dn = torch.empty(nb // 4, dtype=torch.int32, device="cuda")
    s_up, s_dn = torch.cuda.Stream(), torch.cuda.Stream()
    ms = []
    for _ in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s_up):
            d_up.copy_(h_up, non_blocking=True)
        with torch.cuda.stream(s_dn):
            h_dn.copy_(d_dn, non_blocking=True)
        torch.cuda.synchronize()
        ms.append(time.perf_counter() - t0)
    link = 2 * nb / min(ms[1:]) / 1e9
    del h_up, h_dn, d_up, d_dn
    res["host_link"] = {"GB_s_both_ways": round(link, 1), "bytes_per_request_mean": int(bytes_req),
                        "bound_rps": round(link * 1e9 / bytes_req, 1)}
    # host: every request uploads its ciphertexts and reads its results back (link-bound);
    # resident: ciphertexts and results stay in device memory (the serving pattern's resident
    # residues), so the rate is the device's and the loop's
    # native: the same resident groups with the request loop in native code (hefx_serve_run)
    for mode, rates in (("native_resident", (6400, 25600, 51200, 102400, 204800, 409600)),
                        ("grouped_resident", (1600, 6400, 25600, 51200, 102400, 204800)),
                        ("grouped", (100, 400, 1600, 6400, 25600, 51200)), ("per_request", (6400, 25600))):
        ex = GpuExecutor(ctx, nstreams=8, grouped=mode != "per_request", resident=mode.endswith("resident"))
        run = serve_native if mode.startswith("native") else serve
        try:
            out = {}
            for rate in rates:
                count = int(min(2000, max(120, 0.15 * rate)))  # about 0.15 s of arrivals, at least 120
                reqs = poisson_requests(inputs_seed(5, rate), count, rate)
                for r in reqs:
                    ex.warm(r.logn, r.L)
                run(reqs[:8], ex)  # warm kernels on this request mix
                reqs = poisson_requests(inputs_seed(5, rate), count, rate)
                st = run(reqs, ex, budget_bytes=40 << 30)
                out[f"rate_{rate}"] = {k: (round(v, 3) if isinstance(v, float) else v) for k, v in st.items()}
            res[mode] = out
        finally:
            ex.close()
    return res


def inputs_seed(*parts):
    from paper_2501_07047_gb300 import inputs
    return inputs.derive_seed(*parts)


def tensor_flops_per_limb_ntt(log2r: int = 0, log2r2: int = 0) -> float:
    """Algorithmic tensor work of one tensor-path limb-NTT (2 flops per digit MAC) for a split."""
    from paper_2501_07047_gb300 import tensor_plan
    return tensor_plan.flops_per_limb_ntt(LOGN, log2r, log2r2)


def tensor_split(log2r: int = 0, log2r2: int = 0):
    from paper_2501_07047_gb300 import tensor_plan
    return tensor_plan.split(LOGN, log2r, log2r2)


def profile_traffic(kernel: str, which: str):
    """DRAM bytes per launch of the `which` ("fwd" / "inv") kernel from the committed ncu
    summary, if it matches the current source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    try:
        kv = dict(ln.split("=", 1) for ln in open(path).read().split("\n") if "=" in ln)
        import hashlib
        src = os.path.join(ROOT, "paper_2501_07047_gb300", "csrc", kv["source"].strip())
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != kv["source_sha"].strip():
            return None
        return int(float(kv["dram_bytes_per_launch_" + which]))
    except Exception:
        return None


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per = []
    # each step is a bounded sample; the whole --steps K --warmup W run stays near two minutes
    step_s = min(args.cpu_seconds, max(1.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        time_oracle(min(1.0, step_s))
    for _ in range(args.steps):
        per.append(time_oracle(step_s))
    value = statistics.median(p["value"] for p in per)
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "limb-NTT/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(UNITS_PER_STEP / value * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "limbs": L, "batch": BATCH, "path": "cpu-oracle",
                   "units_per_step": UNITS_PER_STEP},
        "impl": "reference",
        "cpu_baseline": {"value": round(value, 2), "unit": "limb-NTT/s", "cores": per[0]["cores"],
                         "kind": "oracle", "sample": per[0]["sample"] + " (per step; bounded sample of the workload)"},
        "e2e": {"value": round(value, 2), "unit": "limb-NTT/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hefx", choices=["hefx", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the BConv and batch measurements")
    ap.add_argument("--extras", default=None,
                    help="comma-separated subset of bconv_config3,batch_config4,he_mult,reduction_ablation")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving arrival-rate sweep")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.steps > 5:
            args.cpu_seconds = min(args.cpu_seconds, 30.0 / args.steps)
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
