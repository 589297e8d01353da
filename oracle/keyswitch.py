"""HE-Mult with hybrid key switching and rescale, composed from the oracle's primitives --
TEST INFRASTRUCTURE ONLY (tests/, smoke() and bench's CPU leg may use it).

The paper lists HE-Mult, Relin. and Rescale as the HE operators built from NTT, INTT,
BConv, VecModMul and VecModAdd (App. A, "Compute Pattern of Bottleneck Kernels") and
measures them with dnum-digit hybrid key switching (Sec. V-A; Sec. V-C, "Effects of
Security Parameters"), without printing their formulas.  This module states them as in
textbook RNS-CKKS, step by step, with no fusion:

  tensor product   d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1        (evaluation form, Q)
  ModUp            per digit j (limbs D_j = [j alpha, min(L, (j+1) alpha))):
                   U_j = c on D_j, BConv_{D_j -> rest of Q u P}(c) elsewhere, c = INTT(d2)
  key product      acc_k = sum_j NTT(U_j) o evk_{j,k}                 (evaluation form, Q u P)
  ModDown          ks_k = (x_Q - BConv_{P->Q}(x_P)) P^-1, x = INTT(acc_k)
  add              c_k = d_k + NTT(ks_k)
  Rescale          c'_k = NTT((x_i - x_{L-1}) q_{L-1}^-1), x = INTT(c_k)  (over q_0..q_{L-2})

`keygen` builds a genuine switching key for s^2 (evk_j = (-a_j s + P g_j s^2, a_j) with the
gadget g_j = Qhat_j [Qhat_j^-1]_{Q_j}, no noise) so that tests can check the relation
c'_0 + c'_1 s = (d0 + d1 s + d2 s^2) / q_{L-1} up to a small error.
"""
from __future__ import annotations

import numpy as np

from . import bconv, key_inner_product, moddown, ntt_batch, polymul_batch, rescale


def digit_ranges(L: int, alpha: int):
    """Limb ranges [lo, hi) of the dnum = ceil(L / alpha) digits."""
    return [(lo, min(L, lo + alpha)) for lo in range(0, L, alpha)]


def _mul(x, y, qs):
    q = np.asarray(qs, dtype=np.uint64)[:, None]
    return ((x.astype(np.uint64) * y.astype(np.uint64)) % q).astype(np.uint32)


def _add(x, y, qs):
    q = np.asarray(qs, dtype=np.uint64)[:, None]
    return ((x.astype(np.uint64) + y.astype(np.uint64)) % q).astype(np.uint32)


def modup(c: np.ndarray, qs, ps, alpha: int) -> np.ndarray:
    """c: [L][n] coefficient form over qs -> [dnum][L + K][n]."""
    L, n = c.shape
    qp = list(qs) + list(ps)
    out = np.zeros((len(digit_ranges(L, alpha)), L + len(ps), n), dtype=np.uint32)
    for j, (lo, hi) in enumerate(digit_ranges(L, alpha)):
        src = list(qs[lo:hi])
        out[j, lo:hi] = c[lo:hi]
        if lo > 0:
            out[j, :lo] = bconv(c[lo:hi], src, qs[:lo])
        out[j, hi:] = bconv(c[lo:hi], src, qp[hi:])
    return out


def he_mult(a0, a1, b0, b1, evk, qs, ps, alpha: int) -> dict:
    """Returns every stage: d0, d1, d2, modup, acc, ks, c0, c1 and the rescaled c0r, c1r."""
    qs, ps = list(qs), list(ps)
    qp = qs + ps
    L = len(qs)
    d0 = _mul(a0, b0, qs)
    d1 = _add(_mul(a0, b1, qs), _mul(a1, b0, qs), qs)
    d2 = _mul(a1, b1, qs)
    c = ntt_batch(d2[None], qs, inverse=True)[0]
    U = modup(c, qs, ps, alpha)
    Uhat = ntt_batch(U, qp)
    acc = key_inner_product(Uhat, evk, qp)
    accc = ntt_batch(acc, qp, inverse=True)
    ks = moddown(accc, qs, ps)
    kshat = ntt_batch(ks, qs)
    c0 = _add(d0, kshat[0], qs)
    c1 = _add(d1, kshat[1], qs)
    cc = ntt_batch(np.stack([c0, c1]), qs, inverse=True)
    r = rescale(cc, qs)
    rhat = ntt_batch(r, qs[:L - 1])
    return {"d0": d0, "d1": d1, "d2": d2, "modup": U, "acc": acc, "ks": ks, "c0": c0, "c1": c1,
            "c0r": rhat[0], "c1r": rhat[1]}


def _residues(vals, primes) -> np.ndarray:
    """Signed integer vector -> [len(primes)][n] residues."""
    v = np.asarray(vals, dtype=object)
    return np.array([[int(x) % q for x in v] for q in primes], dtype=np.uint32)


def keygen(s, qs, ps, alpha: int, a_random: np.ndarray) -> np.ndarray:
    """Switching key for s^2 in evaluation form: [dnum][2][L + K][n].
    s: ternary secret (ints); a_random: [dnum][L + K][n] uniform residues (the a_j)."""
    qs, ps = list(qs), list(ps)
    qp = qs + ps
    L, n = len(qs), len(s)
    P = 1
    for p in ps:
        P *= p
    s_r = _residues(s, qp)
    s2 = polymul_batch(s_r[None], s_r[None], qp)[0]
    dn = len(digit_ranges(L, alpha))
    evk = np.zeros((dn, 2, L + len(ps), n), dtype=np.uint32)
    for j, (lo, hi) in enumerate(digit_ranges(L, alpha)):
        a = a_random[j]
        a_s = polymul_batch(a[None], s_r[None], qp)[0]
        b = np.zeros_like(a)
        for l, r in enumerate(qp):
            g = (P % r) if lo <= l < hi else 0  # P * g_j mod r: 1 on the digit's primes, 0 elsewhere
            b[l] = ((r - a_s[l].astype(np.int64)) % r + g * s2[l].astype(np.int64) % r) % r
        evk[j, 0] = ntt_batch(b[None], qp)[0]
        evk[j, 1] = ntt_batch(a[None], qp)[0]
    return evk


def crt(rows, primes):
    """Residue rows [len(primes)][n] -> Python ints in [0, prod primes)."""
    M = 1
    for q in primes:
        M *= q
    out = []
    for c in range(rows.shape[1]):
        x = 0
        for l, q in enumerate(primes):
            Mi = M // q
            x += int(rows[l, c]) * Mi * pow(Mi, -1, q)
        out.append(x % M)
    return out, M


def phase_error(res: dict, s, qs) -> int:
    """max |c'_0 + c'_1 s - round((d0 + d1 s + d2 s^2) / q_{L-1})| (centered mod Q')."""
    qs = list(qs)
    L = len(qs)
    qsr = qs[:L - 1]
    s_q = _residues(s, qs)
    s2 = polymul_batch(s_q[None], s_q[None], qs)[0]
    d = ntt_batch(np.stack([res["d0"], res["d1"], res["d2"]]), qs, inverse=True)
    w = _add(_add(d[0], polymul_batch(d[1][None], s_q[None], qs)[0], qs), polymul_batch(d[2][None], s2[None], qs)[0], qs)
    W, Q = crt(w, qs)
    cr = ntt_batch(np.stack([res["c0r"], res["c1r"]]), qsr, inverse=True)
    m = _add(cr[0], polymul_batch(cr[1][None], s_q[:L - 1][None], qsr)[0], qsr)
    Mv, Qr = crt(m, qsr)
    ql = qs[-1]
    worst = 0
    for a, b in zip(Mv, W):
        e = (a - (b + ql // 2) // ql) % Qr
        worst = max(worst, min(e, Qr - e))
    return worst
