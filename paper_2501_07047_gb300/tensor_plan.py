"""Work accounting of the tensor-core matrix NTT (used for its roofline)."""

# digit split of the layout-invariant matrix NTT (Sec. IV-A / IV-B): data residues < 2^28
# in K_IN digits of 7 bits, constant matrix entries in K_OUT chunks of 6 bits
K_IN, W_IN, K_OUT, W_OUT = 4, 7, 5, 6


def split(logn: int):
    """R x C split of N = 2^logn used by the tensor path."""
    r = logn // 2
    return 1 << r, 1 << (logn - r)


def flops_per_limb_ntt(logn: int) -> float:
    """2 flops per digit multiply-accumulate over both matrix steps:
    step 1 (K_OUT R) x (K_IN R) by (K_IN R) x C, step 3 R x (K_IN C) by (K_IN C) x (K_OUT C)."""
    R, C = split(logn)
    return 2.0 * K_IN * K_OUT * R * C * (R + C)
