"""Batched uneven polynomial products: workload construction around the hefx batch plan.

All jobs of one ring degree N share one parameter set over the limb primes q_0 .. q_{Lmax-1}
(a job with L limbs uses the first L of them), so every size class is one row list on the
device and the whole batch replays as one CUDA graph (`hefx_batch_polymul`).
"""
from __future__ import annotations

import numpy as np
import torch

from . import hefx, inputs


class UnevenBatch:
    """Device buffers, parameter sets and plan for a list of (log2 N, L) job shapes."""

    def __init__(self, ctx: int, shapes, seed: int, lmax: int = 32, path: str = "auto", fill: bool = True):
        self.ctx = ctx
        self.shapes = list(shapes)
        self.primes = inputs.source_primes(lmax)
        self.params = {}
        for logn, _ in self.shapes:
            if logn not in self.params:
                self.params[logn] = hefx.hefx_params_create(ctx, logn, self.primes)
        self.a, self.b, self.c = [], [], []
        for j, (logn, L) in enumerate(self.shapes):
            n = 1 << logn
            if fill:
                ha = inputs.residue_tensor(inputs.derive_seed(seed, j, 0), 1, self.primes[:L], n)[0]
                hb = inputs.residue_tensor(inputs.derive_seed(seed, j, 1), 1, self.primes[:L], n)[0]
                self.a.append(torch.from_numpy(ha.view(np.int32).copy()).cuda())
                self.b.append(torch.from_numpy(hb.view(np.int32).copy()).cuda())
            else:
                self.a.append(torch.zeros((L, n), dtype=torch.int32, device="cuda"))
                self.b.append(torch.zeros((L, n), dtype=torch.int32, device="cuda"))
            self.c.append(torch.empty((L, n), dtype=torch.int32, device="cuda"))
        jobs = [(self.params[logn], L, self.a[j], self.b[j], self.c[j]) for j, (logn, L) in enumerate(self.shapes)]
        self.plan = hefx.hefx_batch_plan_create(ctx, jobs, path)

    def run(self, stream=None):
        hefx.hefx_batch_polymul(self.ctx, self.plan, stream)

    def coeff_limbs(self) -> int:
        return sum(L << logn for logn, L in self.shapes)

    def host_inputs(self, j: int):
        return (self.a[j].cpu().numpy().view(np.uint32), self.b[j].cpu().numpy().view(np.uint32))

    def close(self):
        if self.plan:
            hefx.hefx_batch_plan_destroy(self.plan)
            self.plan = None
        for p in self.params.values():
            hefx.hefx_params_destroy(p)
        self.params = {}
