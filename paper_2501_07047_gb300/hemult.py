"""HE-Mult with hybrid key switching and rescale, composed from hefx C-ABI calls.

The paper measures HE-Mult, Relin. and Rescale (Sec. V-A; dnum-digit hybrid key switching,
Sec. V-C "Effects of Security Parameters") and builds them from NTT, INTT, BConv, VecModMul
and VecModAdd (App. A); it does not print their formulas, which here are textbook RNS-CKKS:

  d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1            tensor product (evaluation form, Q)
  c = INTT(d2) (= INTT(a1 o b1), taken from a1, b1 directly)
  per digit j (limbs D_j, alpha per digit):              ModUp
      U_j = c on D_j, BConv_{D_j -> rest of Q u P}(c) elsewhere, NTT over Q u P
  acc_k = sum_j U_j o evk_{j,k}                           key inner product
  ks_k = ModDown(INTT(acc_k)), c_k = d_k + NTT(ks_k)
  c'_k = NTT(Rescale(INTT(c_k)))                          over q_0 .. q_{L-2}

Every step runs in libhefx's kernels; this module only allocates workspaces and issues the
calls on one stream.  Inputs and outputs are one ciphertext pair in evaluation form.
"""
from __future__ import annotations

from . import hefx


def digit_ranges(L: int, alpha: int):
    """Limb ranges [lo, hi) of the dnum = ceil(L / alpha) key-switching digits."""
    return [(lo, min(L, lo + alpha)) for lo in range(0, L, alpha)]


class HeMult:
    """Parameter sets, basis-conversion plans and workspaces of one shape (N, Q, P, alpha)."""

    def __init__(self, ctx: int, logn: int, qs, ps, alpha: int, ntt_path: str = "cudacore",
                 bconv_path: str = "auto"):
        import torch
        self.torch = torch
        self.ctx, self.logn = ctx, logn
        self.qs, self.ps = [int(q) for q in qs], [int(p) for p in ps]
        self.L, self.K, self.alpha = len(self.qs), len(self.ps), alpha
        if self.L < 2:
            raise ValueError("HE-Mult with rescale needs at least 2 ciphertext limbs")
        self.digits = digit_ranges(self.L, alpha)
        self.dnum = len(self.digits)
        self.ntt_path, self.bconv_path = ntt_path, bconv_path
        self.pQ = hefx.hefx_params_create(ctx, logn, self.qs)
        self.pQr = hefx.hefx_params_create(ctx, logn, self.qs[:-1])
        self.pQP = hefx.hefx_params_create(ctx, logn, self.qs + self.ps)
        qp = self.qs + self.ps
        # ModUp: one launch for every digit on the CUDA cores ("auto", "cudacore"), or two
        # conversions per digit through hefx_basis_convert on the requested path
        self.modup = hefx.hefx_modup_plan_create(ctx, logn, self.qs, self.ps, alpha) \
            if bconv_path in ("auto", "cudacore") else None
        self.plans = []
        for lo, hi in ([] if self.modup else self.digits):
            src = self.qs[lo:hi]
            lo_plan = hefx.hefx_bconv_plan_create(ctx, logn, src, self.qs[:lo]) if lo > 0 else None
            hi_plan = hefx.hefx_bconv_plan_create(ctx, logn, src, qp[hi:])
            self.plans.append((lo_plan, hi_plan))
        self.plan_pq = hefx.hefx_bconv_plan_create(ctx, logn, self.ps, self.qs)
        n, L, K = 1 << logn, self.L, self.K
        dev = "cuda"
        self.d = torch.empty((3, L, n), dtype=torch.int32, device=dev)
        self.c = torch.empty((L, n), dtype=torch.int32, device=dev)
        self.U = torch.empty((self.dnum, L + K, n), dtype=torch.int32, device=dev)
        self.acc = torch.empty((2, L + K, n), dtype=torch.int32, device=dev)
        self.ks = torch.empty((2, L, n), dtype=torch.int32, device=dev)
        self.cc = torch.empty((2, L, n), dtype=torch.int32, device=dev)

    def close(self) -> None:
        if self.modup:
            hefx.hefx_modup_plan_destroy(self.modup)
        for lo_plan, hi_plan in self.plans:
            if lo_plan:
                hefx.hefx_bconv_plan_destroy(lo_plan)
            hefx.hefx_bconv_plan_destroy(hi_plan)
        hefx.hefx_bconv_plan_destroy(self.plan_pq)
        for p in (self.pQ, self.pQr, self.pQP):
            hefx.hefx_params_destroy(p)

    def launches(self, rescale: bool = True) -> int:
        """Kernel launches of one run (CUDA-core NTT path)."""
        modup = 1 if self.modup else sum(2 if lo else 1 for lo, _ in self.digits)
        return 1 + 1 + modup + 1 + 1 + 1 + 1 + 1 + 1 + (2 if rescale else 0)

    def run(self, a0, a1, b0, b1, evk, out, stream=None, rescale: bool = True) -> None:
        """a*, b*: [L][N] evaluation form over Q; evk: [dnum][2][L+K][N] evaluation form over
        Q u P.  With rescale, out [2][L-1][N] receives (c'_0, c'_1); without, out [2][L][N]
        receives the relinearised (c_0, c_1) over Q.  Copies (c <- d2, and U_j <- c on D_j
        when ModUp runs as per-digit conversions) are device-to-device on the same stream."""
        torch = self.torch
        ctx, s = self.ctx, stream
        d0, d1, d2 = self.d[0], self.d[1], self.d[2]
        st = torch.cuda.current_stream() if s is None else s
        with torch.cuda.stream(st):
            if self.ntt_path == "cudacore":
                # d2 = a1 o b1 only feeds c = INTT(d2): the inverse transform multiplies a1 and
                # b1 as it loads them, and the tensor product writes d0 and d1 only
                hefx.hefx_tensor_product(ctx, self.pQ, a0, a1, b0, b1, d0, d1, None, 1, st)
                hefx.hefx_ntt_inv_hadamard(ctx, self.pQ, a1, b1, self.c, 1, st)
            else:
                hefx.hefx_tensor_product(ctx, self.pQ, a0, a1, b0, b1, d0, d1, d2, 1, st)
                self.c.copy_(d2)
                hefx.hefx_ntt_inv(ctx, self.pQ, self.c, 1, self.ntt_path, st)
            if self.modup:
                hefx.hefx_mod_up(ctx, self.modup, self.c, self.U, 1, st)
            for j, ((lo, hi), (lo_plan, hi_plan)) in enumerate(zip(self.digits, self.plans)):
                self.U[j, lo:hi].copy_(self.c[lo:hi])
                if lo_plan:
                    hefx.hefx_basis_convert(ctx, lo_plan, self.c[lo:hi], self.U[j, :lo], 1, self.bconv_path, st)
                hefx.hefx_basis_convert(ctx, hi_plan, self.c[lo:hi], self.U[j, hi:], 1, self.bconv_path, st)
            hefx.hefx_ntt_fwd(ctx, self.pQP, self.U, self.dnum, self.ntt_path, st)
            hefx.hefx_key_inner_product(ctx, self.pQP, self.U, evk, self.acc, self.dnum, 1, st)
            hefx.hefx_ntt_inv(ctx, self.pQP, self.acc, 2, self.ntt_path, st)
            hefx.hefx_mod_down(ctx, self.plan_pq, self.acc, self.ks, 2, st)
            hefx.hefx_ntt_fwd(ctx, self.pQ, self.ks, 2, self.ntt_path, st)
            dst = self.cc if rescale else out
            # (c_0, c_1) = (d_0, d_1) + (ks_0, ks_1): both halves are contiguous, one launch
            hefx.hefx_vec_mod_add(ctx, self.pQ, self.d[0:2], self.ks, dst, 2, st)
            if rescale:
                self.rescale(self.cc, out, st)

    def rescale(self, c, out, stream=None) -> None:
        """c: [2][L][N] evaluation form over Q (overwritten) -> out [2][L-1][N] evaluation form
        over q_0 .. q_{L-2}: NTT(Rescale(INTT(c))); on the CUDA-core path the rescale runs on
        the forward transform's input load (two launches)."""
        st = self.torch.cuda.current_stream() if stream is None else stream
        with self.torch.cuda.stream(st):
            hefx.hefx_ntt_inv(self.ctx, self.pQ, c, 2, self.ntt_path, st)
            if self.ntt_path == "cudacore":
                hefx.hefx_rescale_ntt(self.ctx, self.pQ, c, out, 2, st)
            else:
                hefx.hefx_rescale(self.ctx, self.pQ, c, out, 2, st)
                hefx.hefx_ntt_fwd(self.ctx, self.pQr, out, 2, self.ntt_path, st)

    def capture(self, a0, a1, b0, b1, evk, out, rescale: bool = True):
        """Records one run on fixed buffers as a CUDA graph (one graph launch replays all the
        kernel launches and copies, removing the host's per-call submission time).  A first
        eager run sets every kernel's attributes and occupancy before the capture.  Returns
        the torch.cuda.CUDAGraph; call .replay() to rerun on the same buffers."""
        torch = self.torch
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.run(a0, a1, b0, b1, evk, out, side, rescale)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(a0, a1, b0, b1, evk, out, torch.cuda.current_stream(), rescale)
        return g

    def stages(self) -> dict:
        """The workspaces after a run (for stage-by-stage parity tests)."""
        return {"d0": self.d[0], "d1": self.d[1], "d2_coeff": self.c, "modup_eval": self.U, "acc_coeff": self.acc,
                "ks_eval": self.ks, "c_coeff": self.cc}
