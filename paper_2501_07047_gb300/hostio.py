"""Transforms of host-resident data with the host<->device copies overlapped.

A caller whose polynomials live in (pinned) host memory pays a copy in and a copy out per
call.  `NttRoundTrip` moves a [batch][L][N] batch in chunks of polynomials over three CUDA
streams (copy in, transform, copy out) and three device buffers, so that while chunk i is
transformed, chunk i + 1 is uploaded and chunk i - 1 downloaded.  The transforms are hefx's
C-ABI calls; this module only orders copies and launches with events.
"""
from __future__ import annotations

from . import hefx


class NttRoundTrip:
    """Forward then inverse NTT of host batches (a round trip, as the bench's end-to-end step),
    or only the forward / inverse transform (`ops`)."""

    NBUF = 3

    def __init__(self, ctx: int, params: int, nlimbs: int, n: int, chunk: int = 8, path: str = "cudacore",
                 ops=("fwd", "inv")):
        """chunk: polynomials per transform launch.  Launches of a few polynomials underfill the
        GPU (at N = 2^16, L = 24 one polynomial per chunk took 0.49 ms per 8-polynomial step
        against 0.31 ms with whole 8-polynomial chunks, which overlap across calls instead)."""
        import torch
        self.torch = torch
        self.ctx, self.params, self.path, self.ops = ctx, params, path, tuple(ops)
        self.chunk = chunk
        self.bufs = [torch.empty((chunk, nlimbs, n), dtype=torch.int32, device="cuda") for _ in range(self.NBUF)]
        self.s_in, self.s_op, self.s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        self.ev_in = [torch.cuda.Event() for _ in range(self.NBUF)]
        self.ev_op = [torch.cuda.Event() for _ in range(self.NBUF)]
        self.ev_free = [torch.cuda.Event() for _ in range(self.NBUF)]
        self.used = [False] * self.NBUF
        self.k = 0  # chunks issued so far (buffer rotation continues across calls)

    def run(self, h_in, h_out) -> None:
        """h_in, h_out: pinned int32 host tensors [batch][L][N] (h_out may be h_in).  Issues
        everything asynchronously after the current stream's work; call `join()` (or
        synchronize) before reading h_out."""
        torch = self.torch
        self.s_in.wait_stream(torch.cuda.current_stream())
        batch = h_in.shape[0]
        for c0 in range(0, batch, self.chunk):
            m = min(self.chunk, batch - c0)
            b = self.k % self.NBUF
            buf = self.bufs[b][:m]
            if self.used[b]:
                self.s_in.wait_event(self.ev_free[b])  # its previous download has finished
            with torch.cuda.stream(self.s_in):
                buf.copy_(h_in[c0:c0 + m], non_blocking=True)
                self.ev_in[b].record(self.s_in)
            self.s_op.wait_event(self.ev_in[b])
            for op in self.ops:
                fn = hefx.hefx_ntt_fwd if op == "fwd" else hefx.hefx_ntt_inv
                fn(self.ctx, self.params, buf, m, self.path, self.s_op)
            self.ev_op[b].record(self.s_op)
            self.s_out.wait_event(self.ev_op[b])
            with torch.cuda.stream(self.s_out):
                h_out[c0:c0 + m].copy_(buf, non_blocking=True)
                self.ev_free[b].record(self.s_out)
            self.used[b] = True
            self.k += 1

    def join(self, stream=None) -> None:
        """Makes `stream` (default: the current stream) wait for every issued chunk."""
        st = self.torch.cuda.current_stream() if stream is None else stream
        st.wait_stream(self.s_out)
