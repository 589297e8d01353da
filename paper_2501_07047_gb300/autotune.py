"""Path tuner: times the CUDA-core and tensor-core paths of a parameter set on the device and
records the faster one as the target of HEFX_PATH_AUTO (`hefx_params_set_auto_path`).

The paper picks the best of three (R, C) splits per HE operator by measurement (Sec. V-A,
"we sweep three (R, C) configurations and report the best-performing one"); hefx generalises
that choice to the path itself.  Results are cached per GPU name and shape in a JSON file
(`$HEFX_TUNE_CACHE`, default ~/.cache/hefx/tune.json).
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import hefx, inputs

CACHE = os.environ.get("HEFX_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "hefx", "tune.json"))


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


def time_paths(ctx: int, params: int, logn: int, primes, batch: int = 4, reps: int = 5) -> dict:
    """Median ms of one forward + inverse NTT of [batch][L][N] per available path."""
    import torch
    n = 1 << logn
    data = inputs.residue_tensor(inputs.derive_seed(90, logn, len(primes)), batch, primes, n)
    d0 = torch.from_numpy(data.view(np.int32).copy()).cuda()
    d = d0.clone()
    s = torch.cuda.current_stream()
    out = {}
    for path in ("cudacore", "tensor"):
        if hefx.raw_status("hefx_ntt_fwd", ctx, params, d.data_ptr(), 0, hefx.PATHS[path], s.cuda_stream) != 0:
            continue
        d.copy_(d0)
        hefx.hefx_ntt_fwd(ctx, params, d, batch, path, s)
        hefx.hefx_ntt_inv(ctx, params, d, batch, path, s)
        torch.cuda.synchronize()
        if not torch.equal(d, d0):
            raise RuntimeError(f"{path}: INTT(NTT(x)) != x while tuning")
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            hefx.hefx_ntt_fwd(ctx, params, d, batch, path, s)
            hefx.hefx_ntt_inv(ctx, params, d, batch, path, s)
            e1.record(s)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        out[path] = float(np.median(ms))
    return out


def tune(ctx: int, params: int, logn: int, primes, use_cache: bool = True) -> str:
    """Chooses the AUTO path of `params` by measurement; returns the chosen path name."""
    import torch
    key = f"{torch.cuda.get_device_name()}|logn={logn}|L={len(primes)}|maxq={max(primes)}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        best = cache[key]["best"]
    else:
        times = time_paths(ctx, params, logn, primes)
        best = min(times, key=times.get)
        cache[key] = {"best": best, "ms": times}
        if use_cache:
            _save_cache(cache)
    hefx.hefx_params_set_auto_path(params, best)
    return best
