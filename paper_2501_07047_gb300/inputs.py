"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle's tests.

This module holds no arithmetic of the method itself (no transform, no reduction, no
basis conversion).  It only produces:

* a counter-based pseudo-random stream (SplitMix64, Steele/Lea/Flood 2014), vectorised
  in numpy with wrapping uint64 arithmetic;
* uniform residues in [0, q) drawn from that stream by rejection sampling;
* lists of NTT-friendly primes (q = 1 mod 2^17, largest first) found with a
  deterministic Miller-Rabin test -- the paper fixes only log2 q = 28 (Sec. V-A) and
  leaves the choice of the moduli open, so these are workload parameters;
* the seeded job and request mixes of the batched and serving workloads.

Both the GPU path and the CPU oracle consume the arrays produced here, so the two sides
never generate their own random inputs.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASK64 = (1 << 64) - 1

BASE_SEED = 0x5EED


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of the SplitMix64 sequence started at `seed`."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & MASK64) + k * _GOLDEN
    return _mix(state)


def derive_seed(*parts: int) -> int:
    """Folds a tuple of integers (config, job, poly, limb, ...) into one 64-bit seed."""
    s = BASE_SEED
    for p in parts:
        s = int(splitmix64((s ^ (int(p) & MASK64)) & MASK64, 1)[0])
    return s


def uniform_residues(seed: int, n: int, q: int) -> np.ndarray:
    """n values uniform in [0, q) as uint32: the top 32 bits of each SplitMix64 output,
    rejected when they fall in the final incomplete block of q."""
    q = int(q)
    assert 1 < q < (1 << 32)
    limit = ((1 << 32) // q) * q
    out = np.empty(0, dtype=np.uint64)
    offset = 0
    while out.size < n:
        want = n - out.size
        chunk = int(want * (1 << 32) / limit) + 64
        v = splitmix64(seed, chunk, offset) >> np.uint64(32)
        offset += chunk
        out = np.concatenate([out, v[v < np.uint64(limit)]])
    return (out[:n] % np.uint64(q)).astype(np.uint32)


def residue_tensor(seed: int, batch: int, primes, n: int) -> np.ndarray:
    """[batch][limb][n] uint32 residues, limb i uniform in [0, primes[i])."""
    primes = list(primes)
    out = np.empty((batch, len(primes), n), dtype=np.uint32)
    for b in range(batch):
        for i, q in enumerate(primes):
            out[b, i] = uniform_residues(derive_seed(seed, b, i), n, q)
    return out


# ----------------------------------------------------------------------------- primes

def _is_prime_u32(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3,215,031,751 (bases 2, 3, 5, 7)."""
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13):
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 3, 5, 7):
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(count: int, bits: int = 28, two_n: int = 1 << 17) -> list[int]:
    """The `count` largest primes below 2^bits with p = 1 (mod two_n), descending.

    With two_n = 2^17 every prime supports negacyclic NTTs of every N <= 2^16."""
    out = []
    k = ((1 << bits) - 1) // two_n
    while len(out) < count and k > 0:
        p = k * two_n + 1
        if p < (1 << bits) and _is_prime_u32(p):
            out.append(p)
        k -= 1
    if len(out) < count:
        raise ValueError(f"only {len(out)} primes of {bits} bits are 1 mod {two_n}")
    return out


def source_primes(count: int) -> list[int]:
    """28-bit ciphertext-modulus limbs q_0, q_1, ... (log2 q = 28 as in Sec. V-A)."""
    return ntt_primes(count, 28)


def special_primes(count: int) -> list[int]:
    """30-bit auxiliary limbs p_0, p_1, ... used as the basis-conversion target."""
    return ntt_primes(count, 30)


# ----------------------------------------------------------------------------- job mixes

def uneven_jobs(seed: int, njobs: int, log2n_choices=(12, 13, 14, 15, 16), lmin=4, lmax=32):
    """Job shapes of the batched uneven workload: (log2 N, limb count) per job."""
    r = splitmix64(seed, 2 * njobs)
    logn = [log2n_choices[int(r[2 * j] % np.uint64(len(log2n_choices)))] for j in range(njobs)]
    limbs = [lmin + int(r[2 * j + 1] % np.uint64(lmax - lmin + 1)) for j in range(njobs)]
    return list(zip(logn, limbs))


def poisson_arrivals(seed: int, count: int, rate_hz: float) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process: exponential gaps from the stream."""
    u = (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    gaps = -np.log1p(-u) / float(rate_hz)
    return np.cumsum(gaps)
