"""Autotuner of the NTT configuration of a parameter set: times every candidate on the device
and records the fastest as what HEFX_PATH_AUTO runs.

Candidates (all bit-exact; checked by INTT(NTT(x)) = x before timing):
  - the CUDA-core radix-2 path, under each of its schedules at N = 2^16 (one launch of 8-CTA
    clusters, or the two-pass column / block schedule; `hefx_params_set_cc_schedule`);
  - the tensor-core matrix NTT for every valid two-factor split N = R x C and the three-factor
    splits R1 x R2 x R3 with the fewest digit MACs (`tensor_plan.tuned_splits`: the paper sweeps
    its (R, C) configurations per operator and keeps the best, Sec. V-A), each with both GEMM
    tile widths (64 or 32 outputs per tile).
The winner is applied with `hefx_params_set_auto_path` and, for the tensor path,
`hefx_params_set_tensor_config` (for the CUDA-core path, `hefx_params_set_cc_schedule`).  Results are cached per GPU name, shape and batch in a JSON
file (`$HEFX_TUNE_CACHE`, default ~/.cache/hefx/tune.json).
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import hefx, inputs, tensor_plan

CACHE = os.environ.get("HEFX_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "hefx", "tune.json"))
TILES = (64, 32)


def _load_cache() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _save_cache(c: dict) -> None:
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except OSError:
        pass


CC_SCHEDULES = {0: "auto", 1: "cluster", 2: "two_pass"}


def candidates(logn: int) -> list:
    """Every configuration the tuner tries at N = 2^logn: ("cudacore", schedule, 0, 0) for each
    CUDA-core schedule built at this size (1 cluster, 2 two-pass; 0 the library's own choice
    where there is no alternative) and ("tensor", log2 R1, log2 R2, tile) for each tuned split
    (two factors: log2 R2 = 0) and tile width."""
    out = [("cudacore", 1, 0, 0), ("cudacore", 2, 0, 0)] if logn == 16 else [("cudacore", 0, 0, 0)]
    for log2r, log2r2 in tensor_plan.tuned_splits(logn):
        for tile in TILES:
            out.append(("tensor", log2r, log2r2, tile))
    return out


def apply(ctx: int, params: int, cand) -> None:
    path, log2r, log2r2, tile = cand
    if path == "tensor":
        hefx.hefx_params_set_tensor_config(ctx, params, log2r, tile, log2r2)
    else:
        hefx.hefx_params_set_cc_schedule(ctx, params, CC_SCHEDULES[log2r])
    hefx.hefx_params_set_auto_path(params, path)


def time_candidates(ctx: int, params: int, logn: int, primes, batch: int = 4, reps: int = 5) -> dict:
    """Median ms of one forward + inverse NTT of [batch][L][N] per available candidate, keyed
    "path/log2r/log2r2/tile"."""
    import torch
    n = 1 << logn
    data = inputs.residue_tensor(inputs.derive_seed(90, logn, len(primes)), batch, primes, n)
    d0 = torch.from_numpy(data.view(np.int32).copy()).cuda()
    d = d0.clone()
    s = torch.cuda.current_stream()
    out = {}
    for cand in candidates(logn):
        path = cand[0]
        if hefx.raw_status("hefx_ntt_fwd", ctx, params, d.data_ptr(), 0, hefx.PATHS[path], s.cuda_stream) != 0:
            continue
        try:
            if path == "tensor":
                hefx.hefx_params_set_tensor_config(ctx, params, cand[1], cand[3], cand[2])
            else:
                hefx.hefx_params_set_cc_schedule(ctx, params, CC_SCHEDULES[cand[1]])
        except hefx.HefxError:
            continue  # not built for this parameter set (e.g. a split 30-bit moduli cannot take)
        d.copy_(d0)
        hefx.hefx_ntt_fwd(ctx, params, d, batch, path, s)
        hefx.hefx_ntt_inv(ctx, params, d, batch, path, s)
        torch.cuda.synchronize()
        if not torch.equal(d, d0):
            raise RuntimeError(f"{cand}: INTT(NTT(x)) != x while tuning")
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            hefx.hefx_ntt_fwd(ctx, params, d, batch, path, s)
            hefx.hefx_ntt_inv(ctx, params, d, batch, path, s)
            e1.record(s)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        out[key_of(cand)] = float(np.median(ms))
    return out


def key_of(cand) -> str:
    return "/".join(str(x) for x in cand)


def parse(key: str):
    path, log2r, log2r2, tile = key.split("/")
    return path, int(log2r), int(log2r2), int(tile)


def tune(ctx: int, params: int, logn: int, primes, batch: int = 4, use_cache: bool = True) -> str:
    """Chooses what HEFX_PATH_AUTO runs for `params` by measurement (or from the cache) and
    applies it; returns the chosen path name."""
    import torch
    key = f"{torch.cuda.get_device_name()}|logn={logn}|L={len(primes)}|maxq={max(primes)}|batch={batch}"
    cache = _load_cache() if use_cache else {}
    if key in cache and "config" in cache[key]:
        best = cache[key]["config"]
    else:
        times = time_candidates(ctx, params, logn, primes, batch)
        best = min(times, key=times.get)
        cache[key] = {"config": best, "ms": times}
        if use_cache:
            _save_cache(cache)
    cand = parse(best)
    apply(ctx, params, cand)
    return cand[0]
