"""Big-integer CRT helpers for pinning the basis conversion -- TEST INFRASTRUCTURE ONLY.

Pure Python integers, no reduction tricks: used to check the oracle's basis conversion
(App. B) against the exact integer it is meant to approximate.
"""
from __future__ import annotations

from math import prod


def crt(residues, moduli) -> int:
    """The unique x in [0, Q) with x = r_i (mod m_i), by the textbook CRT formula."""
    Q = prod(int(m) for m in moduli)
    x = 0
    for r, m in zip(residues, moduli):
        m = int(m)
        qhat = Q // m
        x += int(r) * qhat * pow(qhat, -1, m)
    return x % Q


def fast_conversion_integer(residues, moduli) -> int:
    """y = sum_i [r_i * qhat_i^-1]_{q_i} * qhat_i -- the integer that the fast conversion of
    App. B reduces mod each target prime (no correction of the multiple of Q)."""
    Q = prod(int(m) for m in moduli)
    y = 0
    for r, m in zip(residues, moduli):
        m = int(m)
        qhat = Q // m
        y += (int(r) * pow(qhat, -1, m) % m) * qhat
    return y


def centered(x: int, Q: int) -> int:
    """The representative of x mod Q in (-Q/2, Q/2] (Q odd: [-(Q-1)/2, (Q-1)/2])."""
    x %= Q
    return x - Q if 2 * x > Q else x


def bconv_exact(a, qs, ps):
    """Exact basis conversion of the centered CRT value: out[j][c] = centered(CRT(a[:, c])) mod
    p_j.  a: [L][n] residues (numpy or lists) -> list of Lp lists.  The u-corrected variant of
    the App. B conversion; the centered representative is the reading taken (the paper prints
    only the fast conversion)."""
    Q = prod(int(q) for q in qs)
    n = len(a[0])
    out = [[0] * n for _ in ps]
    for c in range(n):
        x = centered(crt([a[i][c] for i in range(len(qs))], qs), Q)
        for j, p in enumerate(ps):
            out[j][c] = x % int(p)
    return out
