"""hefx oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow CPU statements of what the hefx hot path computes (arXiv 2501.07047,
"CROSS"): the negacyclic NTT / INTT by their definition, the polynomial product, the
basis conversion of App. B and the modular matrix product of Alg. 2.  The arithmetic
lives in `hefx_oracle.c` (64-bit values, 128-bit products, `%` only) and in the pure
Python modules `crt` (big-integer CRT) and `bat` (the BAT constructions of Alg. 2 and
Alg. 5, used to pin the reading of BAT, not by the GPU path).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
package.  It shares no code with the CUDA library and never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hefx_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc into oracle/liboracle.so (plain -O2, no tuning)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, i32, sz = ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t
        lib.or_powmod.restype = u64
        lib.or_powmod.argtypes = [u64, u64, u64]
        lib.or_is_prime.restype = i32
        lib.or_is_prime.argtypes = [u64]
        lib.or_primitive_root.restype = u64
        lib.or_primitive_root.argtypes = [u64]
        lib.or_psi.restype = u64
        lib.or_psi.argtypes = [u64, u64]
        lib.or_inverse.restype = u64
        lib.or_inverse.argtypes = [u64, u64]
        lib.or_bitrev.restype = ctypes.c_uint32
        lib.or_bitrev.argtypes = [ctypes.c_uint32, i32]
        lib.or_ntt_direct_at.restype = ctypes.c_uint32
        lib.or_ntt_direct_at.argtypes = [i32, u64, u64, _u32p, ctypes.c_uint32]
        lib.or_intt_direct_at.restype = ctypes.c_uint32
        lib.or_intt_direct_at.argtypes = [i32, u64, u64, _u32p, ctypes.c_uint32]
        lib.or_ntt_direct.argtypes = [i32, u64, u64, _u32p, _u32p]
        lib.or_ntt_fwd.argtypes = [i32, u64, u64, _u32p]
        lib.or_ntt_inv.argtypes = [i32, u64, u64, _u32p]
        lib.or_ntt_rows.argtypes = [i32, i32, sz, _u32p, _u32p]
        lib.or_polymul_schoolbook.argtypes = [i32, u64, _u32p, _u32p, _u32p]
        lib.or_polymul_ntt.argtypes = [i32, u64, u64, _u32p, _u32p, _u32p]
        lib.or_polymul_rows.argtypes = [i32, sz, _u32p, _u32p, _u32p, _u32p]
        lib.or_bconv.argtypes = [sz, i32, _u32p, i32, _u32p, _u32p, _u32p]
        lib.or_modmatmul.argtypes = [sz, sz, sz, u64, _u32p, _u32p, _u32p]
        lib.or_moddown.argtypes = [sz, i32, _u32p, i32, _u32p, _u32p, _u32p]
        lib.or_rescale.argtypes = [sz, i32, _u32p, _u32p, _u32p]
        lib.or_key_inner_product.argtypes = [sz, i32, _u32p, i32, _u32p, _u32p, _u32p]
        for fn in ("or_ntt_direct", "or_ntt_fwd", "or_ntt_inv", "or_ntt_rows", "or_polymul_schoolbook",
                   "or_polymul_ntt", "or_polymul_rows", "or_bconv", "or_modmatmul"):
            getattr(lib, fn).restype = None
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u32p)


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _logn(n: int) -> int:
    logn = int(n).bit_length() - 1
    assert n == 1 << logn, "N must be a power of two"
    return logn


# ------------------------------------------------------------------ scalar helpers

def powmod(a: int, e: int, q: int) -> int:
    return int(_load().or_powmod(a, e, q))


def is_prime(n: int) -> bool:
    return bool(_load().or_is_prime(n))


def primitive_root(q: int) -> int:
    return int(_load().or_primitive_root(q))


def psi(q: int, n: int) -> int:
    """Primitive 2N-th root of unity g^((q-1)/2N), g the smallest generator of Z_q^*."""
    return int(_load().or_psi(q, n))


def inverse(a: int, q: int) -> int:
    return int(_load().or_inverse(a, q))


def bitrev(x: int, bits: int) -> int:
    return int(_load().or_bitrev(x, bits))


# ------------------------------------------------------------------ transforms

def ntt_direct(a, q: int) -> np.ndarray:
    """O(N^2) forward NTT by the definition (bit-reversed output)."""
    a = _u32(a)
    out = np.empty_like(a)
    _load().or_ntt_direct(_logn(a.size), q, psi(q, a.size), _p(a), _p(out))
    return out


def ntt_at(a, q: int, p: int) -> int:
    """Forward NTT output p by the definition, O(N) (for sampled checks at large N)."""
    a = _u32(a)
    return int(_load().or_ntt_direct_at(_logn(a.size), q, psi(q, a.size), _p(a), p))


def intt_at(ahat, q: int, j: int) -> int:
    """Inverse NTT output j by the definition, O(N log q)."""
    ahat = _u32(ahat)
    return int(_load().or_intt_direct_at(_logn(ahat.size), q, psi(q, ahat.size), _p(ahat), j))


def ntt(a, q: int) -> np.ndarray:
    """Forward negacyclic NTT, natural order in, bit-reversed order out (O(N log N))."""
    a = _u32(a).copy()
    _load().or_ntt_fwd(_logn(a.size), q, psi(q, a.size), _p(a))
    return a


def intt(ahat, q: int) -> np.ndarray:
    """Inverse negacyclic NTT, bit-reversed order in, natural order out."""
    a = _u32(ahat).copy()
    _load().or_ntt_inv(_logn(a.size), q, psi(q, a.size), _p(a))
    return a


def ntt_batch(data: np.ndarray, primes, inverse: bool = False) -> np.ndarray:
    """[batch][L][N] array, limb l modulo primes[l]; returns a new array."""
    d = _u32(data).copy()
    B, L, n = d.shape
    qs = _u32(np.tile(np.asarray(primes, dtype=np.uint32), B))
    assert qs.size == B * L
    _load().or_ntt_rows(_logn(n), int(inverse), B * L, _p(qs), _p(d))
    return d


def polymul_schoolbook(a, b, q: int) -> np.ndarray:
    a, b = _u32(a), _u32(b)
    c = np.empty_like(a)
    _load().or_polymul_schoolbook(_logn(a.size), q, _p(a), _p(b), _p(c))
    return c


def polymul(a, b, q: int) -> np.ndarray:
    a, b = _u32(a), _u32(b)
    c = np.empty_like(a)
    _load().or_polymul_ntt(_logn(a.size), q, psi(q, a.size), _p(a), _p(b), _p(c))
    return c


def polymul_batch(a: np.ndarray, b: np.ndarray, primes) -> np.ndarray:
    a, b = _u32(a), _u32(b)
    B, L, n = a.shape
    c = np.empty_like(a)
    qs = _u32(np.tile(np.asarray(primes, dtype=np.uint32), B))
    _load().or_polymul_rows(_logn(n), B * L, _p(qs), _p(a), _p(b), _p(c))
    return c


def bconv(a: np.ndarray, qs, ps) -> np.ndarray:
    """Basis conversion of App. B.  a: [L][n] (or [batch][L][n]) -> [Lp][n] (or batched)."""
    a = _u32(a)
    qs_a, ps_a = _u32(qs), _u32(ps)
    if a.ndim == 3:
        return np.stack([bconv(x, qs, ps) for x in a])
    L, n = a.shape
    out = np.empty((ps_a.size, n), dtype=np.uint32)
    _load().or_bconv(n, L, _p(qs_a), ps_a.size, _p(ps_a), _p(a), _p(out))
    return out


def modmatmul(A, B, q: int) -> np.ndarray:
    """Z = A @ B mod q (A: H x V, B: V x W)."""
    A, B = _u32(A), _u32(B)
    H, V = A.shape
    V2, W = B.shape
    assert V == V2
    Z = np.empty((H, W), dtype=np.uint32)
    _load().or_modmatmul(H, V, W, q, _p(A), _p(B), _p(Z))
    return Z


def moddown(x: np.ndarray, qs, ps) -> np.ndarray:
    """ModDown: x [L + K][n] (Q limbs, then P limbs), coefficient form -> [L][n]:
    (x_Q - BConv_{P->Q}(x_P)) * P^-1 mod q_j.  Batched over a leading axis."""
    x = _u32(x)
    if x.ndim == 3:
        return np.stack([moddown(v, qs, ps) for v in x])
    qs_a, ps_a = _u32(qs), _u32(ps)
    assert x.shape[0] == qs_a.size + ps_a.size
    out = np.empty((qs_a.size, x.shape[1]), dtype=np.uint32)
    _load().or_moddown(x.shape[1], qs_a.size, _p(qs_a), ps_a.size, _p(ps_a), _p(x), _p(out))
    return out


def rescale(x: np.ndarray, qs) -> np.ndarray:
    """Rescale: x [L][n] coefficient form over qs -> [L-1][n]: (x_i - x_{L-1}) q_{L-1}^-1 mod q_i."""
    x = _u32(x)
    if x.ndim == 3:
        return np.stack([rescale(v, qs) for v in x])
    qs_a = _u32(qs)
    assert x.shape[0] == qs_a.size >= 2
    out = np.empty((qs_a.size - 1, x.shape[1]), dtype=np.uint32)
    _load().or_rescale(x.shape[1], qs_a.size, _p(qs_a), _p(x), _p(out))
    return out


def key_inner_product(digits: np.ndarray, evk: np.ndarray, qs) -> np.ndarray:
    """sum_j digits[j] o evk[j][k] mod q per limb: digits [dnum][nl][n], evk [dnum][2][nl][n]
    -> [2][nl][n]."""
    digits, evk, qs_a = _u32(digits), _u32(evk), _u32(qs)
    dnum, nl, n = digits.shape
    assert evk.shape == (dnum, 2, nl, n) and qs_a.size == nl
    out = np.empty((2, nl, n), dtype=np.uint32)
    _load().or_key_inner_product(n, nl, _p(qs_a), dnum, _p(digits), _p(evk), _p(out))
    return out
