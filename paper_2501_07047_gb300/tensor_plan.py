"""Work accounting of the tensor-core matrix NTT (used for its roofline)."""

# digit split of the layout-invariant matrix NTT (Sec. IV-A / IV-B) as run by the pipelined
# tensor kernels: data residues < 2^28 in K_IN digits of 7 bits, constants in K_OUT chunks of
# 7 bits (partial sums below 2^24, exact in fp32)
K_IN, W_IN, K_OUT, W_OUT = 4, 7, 4, 7


def split(logn: int, log2r: int = 0):
    """R x C split of N = 2^logn used by the tensor path (log2r = 0: the default, R =
    2^floor(logn / 2))."""
    r = log2r or logn // 2
    return 1 << r, 1 << (logn - r)


def splits(logn: int) -> list:
    """log2 R of every split the tensor path accepts at N = 2^logn: both factors 128 or 256
    (128-row data blocks; exact fp32 sums of 7-bit digit products need reduction lengths of at
    most 256: 4 * 256 * 127 * 127 < 2^24)."""
    return [r for r in (7, 8) if 7 <= logn - r <= 8]


def flops_per_limb_ntt(logn: int, log2r: int = 0) -> float:
    """2 flops per digit multiply-accumulate over both matrix steps:
    step 1 (R data columns of K_IN R digits) by (K_OUT R) constant rows, step 3 likewise with C."""
    R, C = split(logn, log2r)
    return 2.0 * K_IN * K_OUT * R * C * (R + C)


def flops_per_step_launch(logn: int, limbs: int) -> float:
    """Flops of one GEMM launch (one matrix step) over `limbs` limb-NTTs (square split)."""
    return flops_per_limb_ntt(logn) / 2 * limbs
