"""Host check of the BAT lazy modular reduction's identity (the paper's appendix "BAT for
Modular Reduction"): with psum = sum_j c_j 2^(8j) (bytes c_j) and LC_j = 2^(8(4+j)) mod q split
into bytes LC_{j,k},

    low + sum_k (sum_j c_{4+j} LC_{j,k}) 2^(8k)  ==  psum  (mod q),

where low = psum mod 2^32, each inner sum < 2^24 (exact in fp32), and the merged value
< 2^44.  Exact Python integers; a dropped high byte, a wrong shift or a transposed LC fails."""
import random

import pytest

from paper_2501_07047_gb300 import inputs


def bat_lazy(psum: int, q: int) -> tuple[int, list[int]]:
    c = [(psum >> (8 * j)) & 255 for j in range(8)]
    lc = [pow(2, 8 * (4 + j), q) for j in range(4)]
    lcb = [[(lc[j] >> (8 * k)) & 255 for k in range(4)] for j in range(4)]
    s = [sum(c[4 + j] * lcb[j][k] for j in range(4)) for k in range(4)]
    low = psum & 0xFFFFFFFF
    return low + sum(s[k] << (8 * k) for k in range(4)), s


@pytest.mark.parametrize("q", list(inputs.source_primes(3)) + list(inputs.special_primes(3)))
def test_identity_and_ranges(q):
    rng = random.Random(q)
    cases = [(q - 1, q - 1), (0, q - 1), (1, 1)] + [(rng.randrange(q), rng.randrange(q)) for _ in range(2000)]
    for x, y in cases:
        psum = x * y
        merged, s = bat_lazy(psum, q)
        assert merged % q == psum % q
        assert all(v < 4 * 255 * 255 < 2 ** 24 for v in s)
        assert merged < 2 ** 44


def test_full_64_bit_psum():
    """Any 64-bit value (not only products of residues) reduces the same way."""
    rng = random.Random(7)
    q = inputs.special_primes(1)[0]
    for _ in range(2000):
        v = rng.getrandbits(64)
        assert bat_lazy(v, q)[0] % q == v % q
