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
