"""Work accounting of the tensor-core matrix NTT (used for its roofline)."""

# digit split of the layout-invariant matrix NTT (Sec. IV-A / IV-B) as run by the pipelined
# tensor kernels: data residues < 2^28 in K_IN digits of 7 bits, constants in K_OUT chunks of
# 7 bits (partial sums below 2^24, exact in fp32); residues of 29-30-bit moduli in digits and
# chunks of W_WIDE = 8 bits, exact for reduction lengths up to MAX_FACTOR_WIDE
K_IN, W_IN, K_OUT, W_OUT = 4, 7, 4, 7
W_WIDE, MAX_FACTOR_WIDE = 8, 64


def split(logn: int, log2r: int = 0, log2r2: int = 0):
    """Factors of N = 2^logn used by the tensor path: (R, C) for two factors (log2r = 0: R =
    2^floor(logn / 2)), (R1, R2, R3) when log2r2 > 0."""
    r = log2r or logn // 2
    if log2r2:
        return 1 << r, 1 << log2r2, 1 << (logn - r - log2r2)
    return 1 << r, 1 << (logn - r)


def splits(logn: int) -> list:
    """(log2r, log2r2) of every split the tensor path accepts at N = 2^logn.
    Two factors: both 64 .. 256 (64-wide transposing digit split; exact fp32 sums of 7-bit
    digit products need reduction lengths of at most 256: 4 * 256 * 127 * 127 < 2^24; a step
    with 64 data rows per limb packs two polynomials into one 128-row block).  Three factors:
    the first 64 .. 256, the others 16 .. 256."""
    two = [(r, 0) for r in (6, 7, 8) if 6 <= logn - r <= 8]
    three = [(a, b) for a in (6, 7, 8) for b in (4, 5, 6, 7, 8) if 4 <= logn - a - b <= 8]
    return two + three


def splits_wide(logn: int) -> list:
    """(log2r, log2r2) of the splits the tensor path accepts for moduli of 29-30 bits: every
    factor at most 64 (4 * 64 * 255 * 255 < 2^24), the first exactly 64."""
    return [(a, b) for a, b in splits(logn) if a == 6 and b <= 6 and logn - a - b <= 6]


def tuned_splits(logn: int) -> list:
    """The splits the autotuner times: every two-factor split, and the three-factor splits with
    the fewest digit MACs (smallest R1 + R2 + R3)."""
    all_ = splits(logn)
    three = [s for s in all_ if s[1]]
    best = min((sum(split(logn, *s)) for s in three), default=None)
    return [s for s in all_ if not s[1]] + [s for s in three if sum(split(logn, *s)) == best]


def flops_per_limb_ntt(logn: int, log2r: int = 0, log2r2: int = 0) -> float:
    """2 flops per digit multiply-accumulate over the matrix steps: a step over a factor f
    takes N / f data rows of K_IN f digits against K_OUT f constant rows, so each step costs
    K_IN K_OUT N f and the transform K_IN K_OUT N (sum of the factors)."""
    return 2.0 * K_IN * K_OUT * (1 << logn) * sum(split(logn, log2r, log2r2))


def flops_per_step_launch(logn: int, limbs: int) -> float:
    """Flops of one GEMM launch (one matrix step) over `limbs` limb-NTTs (square split)."""
    return flops_per_limb_ntt(logn) / 2 * limbs
