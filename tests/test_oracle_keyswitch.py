"""Pins of the oracle's key-switching pieces (ModDown, Rescale, key inner product) and of the
composed HE-Mult, against big-integer arithmetic and the decryption relation of a genuine
switching key.  Definitions: textbook RNS-CKKS for the HE operators the paper measures
(Sec. V-A, V-C; App. A), see oracle/keyswitch.py."""
import numpy as np
import pytest

import oracle
from oracle import keyswitch as ks
from paper_2501_07047_gb300 import inputs


def _crt(rows, primes):
    return ks.crt(np.asarray(rows, dtype=np.uint32), primes)


def _prod(ps):
    P = 1
    for p in ps:
        P *= p
    return P


@pytest.mark.parametrize("L,K", [(3, 2), (5, 4), (2, 1)])
def test_moddown_big_integer(L, K):
    n = 64
    qs, ps = inputs.source_primes(L), inputs.special_primes(K)
    x = inputs.residue_tensor(inputs.derive_seed(40, L, K), 1, list(qs) + list(ps), n)[0]
    out = oracle.moddown(x, qs, ps)
    P = _prod(ps)
    Xs, QP = _crt(x, list(qs) + list(ps))
    got, Q = _crt(out, qs)
    # fast conversion of the P part: Y = sum_k [x_k phat_k^-1]_{p_k} phat_k = (X mod P) + u P
    for c in range(n):
        X = Xs[c]
        Y = sum((int(x[L + k, c]) * pow(P // p, -1, p) % p) * (P // p) for k, p in enumerate(ps))
        u = (Y - X % P) // P
        assert (Y - X % P) % P == 0 and 0 <= u < K
        assert (X - Y) % P == 0
        assert got[c] == ((X - Y) // P) % Q
        assert got[c] == (X // P - u) % Q


def test_moddown_special_cases():
    qs, ps = inputs.source_primes(3), inputs.special_primes(2)
    P = _prod(ps)
    n = 8
    # x = P * z for z < Q: the P limbs are 0, and ModDown returns z exactly
    z = [3, 0, 1, 12345, 2 ** 60 + 7, 5, 9, 11]
    x = np.array([[(P * v) % r for v in z] for r in list(qs) + list(ps)], dtype=np.uint32)
    got, _ = _crt(oracle.moddown(x, qs, ps), qs)
    assert got == z


def test_moddown_planted_sign_fails():
    qs, ps = inputs.source_primes(3), inputs.special_primes(2)
    x = inputs.residue_tensor(inputs.derive_seed(41), 1, list(qs) + list(ps), 16)[0]
    good = oracle.moddown(x, qs, ps)
    # planted mistake on the CPU: x_Q + BConv instead of x_Q - BConv
    y = oracle.bconv(x[3:], ps, qs).astype(np.uint64)
    P = _prod(ps)
    bad = np.array([((x[j].astype(np.uint64) + y[j]) % q * pow(P % q, -1, q)) % q for j, q in enumerate(qs)],
                   dtype=np.uint32)
    assert not np.array_equal(bad, good)


@pytest.mark.parametrize("L", [2, 4, 7])
def test_rescale_is_floor_division(L):
    n = 64
    qs = inputs.source_primes(L)
    x = inputs.residue_tensor(inputs.derive_seed(42, L), 1, qs, n)[0]
    X, _ = _crt(x, qs)
    got, _ = _crt(oracle.rescale(x, qs), qs[:L - 1])
    assert got == [v // qs[-1] for v in X]
    # planted mistake: dividing by q_0 instead of q_{L-1} breaks the relation
    q0 = qs[0]
    bad = np.array([((x[i].astype(np.uint64) + q - x[L - 1] % q) % q * pow(q0 % q, -1, q)) % q
                    if q != q0 else x[i] for i, q in enumerate(qs[:L - 1])], dtype=np.uint32)
    if L > 2:
        assert _crt(bad, qs[:L - 1])[0] != got


def test_key_inner_product_definition():
    qs = list(inputs.source_primes(3)) + list(inputs.special_primes(1))
    dnum, n = 3, 16
    dig = np.stack([inputs.residue_tensor(inputs.derive_seed(43, j), 1, qs, n)[0] for j in range(dnum)])
    evk = np.stack([np.stack([inputs.residue_tensor(inputs.derive_seed(44, j, k), 1, qs, n)[0] for k in range(2)])
                    for j in range(dnum)])
    out = oracle.key_inner_product(dig, evk, qs)
    for k in range(2):
        for l, q in enumerate(qs):
            for c in range(n):
                assert out[k, l, c] == sum(int(dig[j, l, c]) * int(evk[j, k, l, c]) for j in range(dnum)) % q


def _shape(n, L, K, alpha, seed):
    qs, ps = inputs.source_primes(L), inputs.special_primes(K)
    qp = list(qs) + list(ps)
    rng = np.random.default_rng(seed)
    s = rng.integers(-1, 2, n)
    dn = len(ks.digit_ranges(L, alpha))
    a_r = np.stack([inputs.residue_tensor(inputs.derive_seed(seed, 1, j), 1, qp, n)[0] for j in range(dn)])
    evk = ks.keygen(s, qs, ps, alpha, a_r)
    ins = [inputs.residue_tensor(inputs.derive_seed(seed, 2, c), 1, qs, n)[0] for c in range(4)]
    return qs, ps, s, evk, ins


@pytest.mark.parametrize("n,L,K,alpha", [(64, 5, 2, 2), (32, 3, 3, 3), (128, 6, 4, 4)])
def test_he_mult_decrypts(n, L, K, alpha):
    qs, ps, s, evk, ins = _shape(n, L, K, alpha, seed=45 + L)
    res = ks.he_mult(*ins, evk, qs, ps, alpha)
    assert ks.phase_error(res, s, qs) <= 2 * n + 2 * K + 8


def test_he_mult_planted_digit_mistake_fails():
    n, L, K, alpha = 64, 5, 2, 2
    qs, ps, s, evk, ins = _shape(n, L, K, alpha, seed=46)
    orig = ks.digit_ranges
    try:  # planted mistake on the CPU: the second ModUp digit skips its first limb
        ks.digit_ranges = lambda L_, a_: [(lo + 1, hi) if j == 1 else (lo, hi) for j, (lo, hi) in enumerate(orig(L_, a_))]
        bad = ks.he_mult(*ins, evk, qs, ps, alpha)
    finally:
        ks.digit_ranges = orig
    assert ks.phase_error(bad, s, qs) > 10 ** 6
