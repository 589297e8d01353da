"""Work accounting of the tensor-core matrix NTT (used for its roofline)."""

# digit split of the layout-invariant matrix NTT (Sec. IV-A / IV-B) as run by the pipelined
# tensor kernels: data residues < 2^28 in K_IN digits of 7 bits, constants in K_OUT chunks of
# 7 bits (partial sums below 2^24, exact in fp32)
K_IN, W_IN, K_OUT, W_OUT = 4, 7, 4, 7


def split(logn: int):
    """R x C split of N = 2^logn used by the tensor path."""
    r = logn // 2
    return 1 << r, 1 << (logn - r)


def flops_per_limb_ntt(logn: int) -> float:
    """2 flops per digit multiply-accumulate over both matrix steps:
    step 1 (R data columns of K_IN R digits) by (K_OUT R) constant rows, step 3 likewise with C."""
    R, C = split(logn)
    return 2.0 * K_IN * K_OUT * R * C * (R + C)


def flops_per_step_launch(logn: int, limbs: int) -> float:
    """Flops of one GEMM launch (one matrix step) over `limbs` limb-NTTs (square split)."""
    return flops_per_limb_ntt(logn) / 2 * limbs
