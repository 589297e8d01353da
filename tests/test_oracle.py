"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Every check here compares the oracle with something other than itself: hand-computed
cases, closed forms, brute force on tiny inputs, pure-Python big-integer arithmetic and
invariants.  A few checks plant a plausible mistake (a wrong output order, the inverse
root, a cyclic instead of a negacyclic wrap) and assert that the pins reject it.
"""
import os
from math import prod

import numpy as np
import pytest

import oracle
from oracle import bat, crt
from paper_2501_07047_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_small.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, params, inp, exp = [s.strip() for s in line.split("|")]
        kv = dict(p.split("=") for p in params.split())
        rows.append((name, kv, inp, [int(x) for x in exp.split()]))
    return rows


def horner_eval(a, x, q):
    """Independent pure-Python polynomial evaluation."""
    acc = 0
    for c in reversed([int(v) for v in a]):
        acc = (acc * x + c) % q
    return acc


def brv(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


def negacyclic_bigint(a, b, q):
    n = len(a)
    c = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                c[k] += int(a[i]) * int(b[j])
            else:
                c[k - n] -= int(a[i]) * int(b[j])
    return [x % q for x in c]


# ----------------------------------------------------------------------------- parameters

def test_primes_are_ntt_friendly():
    qs = inputs.source_primes(36)
    ps = inputs.special_primes(12)
    assert qs[0] == 268042241 and ps[0] == 1073479681
    assert qs == sorted(qs, reverse=True) and len(set(qs + ps)) == 48
    for q in qs + ps:
        assert oracle.is_prime(q)
        assert (q - 1) % (1 << 17) == 0
    assert all(q < 2**28 for q in qs) and all(2**29 < p < 2**30 for p in ps)
    # nothing between 2^28 - 1 and qs[0] is a prime = 1 mod 2^17 (largest-first rule)
    k = qs[0] + (1 << 17)
    while k < 2**28:
        assert not oracle.is_prime(k)
        k += 1 << 17


def test_is_prime_brute_force():
    for n in range(0, 2000):
        expect = n >= 2 and all(n % d for d in range(2, n))
        assert oracle.is_prime(n) == expect, n


@pytest.mark.parametrize("q", [17, 97, 193, 257, 7681, 12289])
def test_primitive_root_brute_force(q):
    g = oracle.primitive_root(q)
    order = lambda x: next(k for k in range(1, q) if pow(x, k, q) == 1)
    assert order(g) == q - 1
    assert all(order(x) != q - 1 for x in range(2, g))


@pytest.mark.parametrize("q,n", [(17, 4), (97, 16), (7681, 256), (268042241, 4096), (268042241, 65536),
                                 (1073479681, 65536)])
def test_psi_is_primitive_2n_th_root(q, n):
    psi = oracle.psi(q, n)
    assert pow(psi, n, q) == q - 1           # psi^N = -1
    assert pow(psi, 2 * n, q) == 1
    assert psi == pow(oracle.primitive_root(q), (q - 1) // (2 * n), q)
    if (q - 1) % (4 * n) == 0:
        assert oracle.psi(q, 2 * n) ** 2 % q == psi   # tables for different N agree


# ----------------------------------------------------------------------------- NTT

def test_golden_hand_cases():
    for name, kv, inp, exp in _golden():
        if name == "ntt":
            q = int(kv["q"])
            a = [int(x) for x in inp.split()]
            assert list(oracle.ntt(a, q)) == exp
            assert list(oracle.ntt_direct(a, q)) == exp
            assert list(oracle.intt(exp, q)) == a
        elif name == "polymul":
            q = int(kv["q"])
            a, b = ([int(x) for x in s.split()] for s in inp.split(";"))
            assert list(oracle.polymul_schoolbook(a, b, q)) == exp
            assert list(oracle.polymul(a, b, q)) == exp
        elif name == "bconv":
            qs = [int(x) for x in kv["qs"].split(",")]
            ps = [int(x) for x in kv["ps"].split(",")]
            res = np.array([[int(x)] for x in inp.split()], dtype=np.uint32)
            assert list(oracle.bconv(res, qs, ps)[:, 0]) == exp


@pytest.mark.parametrize("logn", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("q", [97, 7681, 268042241, 1073479681])
def test_ntt_direct_equals_evaluation_at_odd_powers(logn, q):
    n = 1 << logn
    if (q - 1) % (2 * n):
        pytest.skip("no 2N-th root")
    a = inputs.uniform_residues(inputs.derive_seed(100, logn, q), n, q)
    psi = oracle.psi(q, n)
    expect = [horner_eval(a, pow(psi, 2 * brv(p, logn) + 1, q), q) for p in range(n)]
    assert list(oracle.ntt_direct(a, q)) == expect
    assert list(oracle.ntt(a, q)) == expect
    assert [oracle.ntt_at(a, q, p) for p in range(n)] == expect


@pytest.mark.parametrize("logn", [3, 6, 10, 12])
def test_ntt_special_inputs(logn):
    q, n = 268042241, 1 << logn
    psi = oracle.psi(q, n)
    delta = np.zeros(n, np.uint32)
    delta[0] = 1
    assert (oracle.ntt(delta, q) == 1).all()                       # NTT(1) = all ones
    x = np.zeros(n, np.uint32)
    x[1] = 1
    assert [int(v) for v in oracle.ntt(x, q)] == [pow(psi, 2 * brv(p, logn) + 1, q) for p in range(n)]
    assert (oracle.ntt(np.zeros(n, np.uint32), q) == 0).all()


def test_ntt_pins_reject_planted_mistakes():
    q, logn = 7681, 4
    n = 1 << logn
    a = inputs.uniform_residues(7, n, q)
    psi = oracle.psi(q, n)
    good = list(oracle.ntt_direct(a, q))
    natural = [horner_eval(a, pow(psi, 2 * p + 1, q), q) for p in range(n)]       # no bit reversal
    inv_root = [horner_eval(a, pow(psi, -(2 * brv(p, logn) + 1), q), q) for p in range(n)]
    omega = psi * psi % q
    cyclic = [horner_eval(a, pow(omega, brv(p, logn), q), q) for p in range(n)]   # x^N - 1 ring
    for wrong in (natural, inv_root, cyclic):
        assert wrong != good


@pytest.mark.parametrize("logn", [3, 7, 12, 16])
def test_intt_inverts_ntt(logn):
    q = inputs.source_primes(3)[2]
    n = 1 << logn
    a = inputs.uniform_residues(inputs.derive_seed(200, logn), n, q)
    ahat = oracle.ntt(a, q)
    assert (oracle.intt(ahat, q) == a).all()
    for j in (0, 1, n // 2, n - 1):
        assert oracle.intt_at(ahat, q, j) == a[j]
    for p in (0, 1, n - 1):
        assert oracle.ntt_at(a, q, p) == ahat[p]


def test_ntt_linearity():
    q, n = 268042241, 1024
    a = inputs.uniform_residues(1, n, q)
    b = inputs.uniform_residues(2, n, q)
    s = ((a.astype(np.uint64) + 5 * b.astype(np.uint64)) % q).astype(np.uint32)
    lhs = oracle.ntt(s, q).astype(np.uint64)
    rhs = (oracle.ntt(a, q).astype(np.uint64) + 5 * oracle.ntt(b, q).astype(np.uint64)) % q
    assert (lhs == rhs).all()


def test_batched_rows_match_single():
    primes = inputs.source_primes(3)
    data = inputs.residue_tensor(3, 2, primes, 256)
    out = oracle.ntt_batch(data, primes)
    back = oracle.ntt_batch(out, primes, inverse=True)
    for b in range(2):
        for l, q in enumerate(primes):
            assert (out[b, l] == oracle.ntt(data[b, l], q)).all()
    assert (back == data).all()


# ----------------------------------------------------------------------------- products

@pytest.mark.parametrize("logn", [1, 2, 3, 5, 7])
def test_schoolbook_vs_bigint(logn):
    q, n = 268042241, 1 << logn
    a = inputs.uniform_residues(11, n, q)
    b = inputs.uniform_residues(12, n, q)
    assert list(oracle.polymul_schoolbook(a, b, q)) == negacyclic_bigint(a, b, q)


@pytest.mark.parametrize("logn,q", [(4, 97), (8, 7681), (10, 268042241), (12, 268042241), (9, 1073479681)])
def test_convolution_theorem(logn, q):
    n = 1 << logn
    a = inputs.uniform_residues(21, n, q)
    b = inputs.uniform_residues(22, n, q)
    assert (oracle.polymul(a, b, q) == oracle.polymul_schoolbook(a, b, q)).all()


def test_polymul_wrap_sign_planted():
    q, n = 97, 8
    a = inputs.uniform_residues(5, n, q)
    b = inputs.uniform_residues(6, n, q)
    cyc = [0] * n
    for i in range(n):
        for j in range(n):
            cyc[(i + j) % n] += int(a[i]) * int(b[j])
    assert list(oracle.polymul_schoolbook(a, b, q)) != [x % q for x in cyc]


# ----------------------------------------------------------------------------- basis conversion

@pytest.mark.parametrize("L,Lp", [(1, 3), (2, 2), (5, 3), (24, 8)])
def test_bconv_bigint_crt(L, Lp):
    qs = inputs.source_primes(L)
    ps = inputs.special_primes(Lp)
    n = 64
    a = np.stack([inputs.uniform_residues(inputs.derive_seed(300, i), n, q) for i, q in enumerate(qs)])
    out = oracle.bconv(a, qs, ps)
    Q = prod(qs)
    for x in range(n):
        res = [int(a[i, x]) for i in range(L)]
        xv = crt.crt(res, qs)
        y = crt.fast_conversion_integer(res, qs)
        assert y % Q == xv
        u = (y - xv) // Q
        assert 0 <= u < L
        for j, p in enumerate(ps):
            assert out[j, x] == y % p
        if L == 1:
            assert [int(out[j, x]) for j in range(Lp)] == [res[0] % p for p in ps]


def test_bconv_zero_and_planted():
    qs, ps = inputs.source_primes(4), inputs.special_primes(2)
    z = np.zeros((4, 8), np.uint32)
    assert (oracle.bconv(z, qs, ps) == 0).all()
    a = np.stack([inputs.uniform_residues(i, 8, q) for i, q in enumerate(qs)])
    out = oracle.bconv(a, qs, ps)
    # planted mistake: dropping the qhat^-1 factor of step 1 changes the result
    Q = prod(qs)
    wrong = [sum(int(a[i, 0]) * (Q // q) for i, q in enumerate(qs)) % ps[0]]
    assert wrong[0] != out[0, 0]


# ----------------------------------------------------------------------------- matmul and BAT

def test_modmatmul_bigint():
    q = 268042241
    A = np.stack([inputs.uniform_residues(i, 7, q) for i in range(5)])
    B = np.stack([inputs.uniform_residues(50 + i, 3, q) for i in range(7)])
    Z = oracle.modmatmul(A, B, q)
    for h in range(5):
        for w in range(3):
            assert Z[h, w] == sum(int(A[h, v]) * int(B[v, w]) for v in range(7)) % q


@pytest.mark.parametrize("w,k_in,w_out,k_out", [(8, 4, 8, 4), (7, 4, 6, 5), (8, 4, 8, 4)])
def test_bat_modmatmul_matches_plain(w, k_in, w_out, k_out):
    q = inputs.source_primes(1)[0]
    A = [[int(x) for x in inputs.uniform_residues(i, 6, q)] for i in range(4)]
    B = [[int(x) for x in inputs.uniform_residues(40 + i, 5, q)] for i in range(6)]
    Z, peak = bat.bat_modmatmul(A, B, q, w, k_in, w_out, k_out)
    assert Z == oracle.modmatmul(np.array(A, np.uint32), np.array(B, np.uint32), q).tolist()
    assert peak <= 6 * k_in * ((1 << w) - 1) * ((1 << w_out) - 1)


def test_bat_scalar_exhaustive_small_q():
    q, a = 65521, 40503   # 16-bit prime, K = 2 byte chunks
    M = bat.direct_scalar_bat(a, q, 8, 2)
    for b in range(1 << 16):
        b0, b1 = b & 255, b >> 8
        psum = [M[i][0] * b0 + M[i][1] * b1 for i in range(2)]
        assert (psum[0] + (psum[1] << 8)) % q == a * b % q


def test_bat_garble_reading():
    """Eqs. (1)-(5) print shift 2^i; with that literal reading the identity fails."""
    q, a, b = 268042241, 123456789, 987654321 % 268042241
    b_chunks = bat.chunk_decompose(b, 8, 4)
    literal = sum(((a << i) % q) * bc for i, bc in enumerate(b_chunks)) % q
    read = sum(((a << (8 * i)) % q) * bc for i, bc in enumerate(b_chunks)) % q
    assert read == a * b % q and literal != a * b % q


@pytest.mark.parametrize("seed", range(6))
def test_iterative_bat_congruent(seed):
    q = inputs.source_primes(4)[seed % 4]
    a = int(inputs.uniform_residues(seed, 1, q)[0])
    M = bat.iterative_scalar_bat(a, q, 8, 4)
    D = bat.direct_scalar_bat(a, q, 8, 4)
    for j in range(4):
        assert all(0 <= M[i][j] < 256 for i in range(4))
        col = sum(M[i][j] << (8 * i) for i in range(4))
        assert col % q == (a << (8 * j)) % q == bat.chunk_merge([D[i][j] for i in range(4)], 8)


# ------------------------------------------------------------------ exact (u-corrected) BConv
def test_bconv_exact_small_signed_values():
    from math import prod
    qs, ps = inputs.source_primes(4), inputs.special_primes(3)
    Q = prod(qs)
    zs = [0, 1, -1, 2, -2, 12345, -98765, 2 ** 40 + 3, -(2 ** 50), (Q - 1) // 2, -(Q - 1) // 2]
    a = [[z % q for z in zs] for q in qs]
    out = crt.bconv_exact(a, qs, ps)
    for j, p in enumerate(ps):
        assert out[j] == [z % p for z in zs]


@pytest.mark.parametrize("L,Lp", [(1, 2), (3, 4), (24, 8)])
def test_bconv_exact_vs_fast_conversion(L, Lp):
    from math import prod
    qs, ps = inputs.source_primes(L), inputs.special_primes(Lp)
    Q = prod(qs)
    a = inputs.residue_tensor(inputs.derive_seed(47, L, Lp), 1, qs, 32)[0]
    exact = crt.bconv_exact(a, qs, ps)
    fast = oracle.bconv(a, qs, ps)
    for c in range(32):
        col = [int(a[i, c]) for i in range(L)]
        y = crt.fast_conversion_integer(col, qs)
        xb = crt.centered(crt.crt(col, qs), Q)
        k = (y - xb) // Q
        assert (y - xb) % Q == 0 and 0 <= k <= L
        for j, p in enumerate(ps):
            assert (int(fast[j, c]) - exact[j][c] - k * Q) % p == 0


def test_ntt_n_2_17_pinned_by_direct_evaluation():
    """The O(N log N) oracle at N = 2^17 (q = 1 mod 2^18) agrees with the per-output
    definition a(psi^(2 brv(p) + 1)) at sampled positions, and INTT inverts it."""
    q = inputs.ntt_primes(1, 30, two_n=1 << 18)[0]
    n = 1 << 17
    a = inputs.residue_tensor(inputs.derive_seed(49), 1, [q], n)[0, 0]
    ahat = oracle.ntt(a, q)
    for pos in [0, 1, 2, 12345, n // 2, n - 1]:
        assert int(ahat[pos]) == oracle.ntt_at(a, q, pos)
    assert (oracle.intt(ahat, q) == a).all()
