"""GPU parity of the RNS basis conversion against the CPU oracle through the C ABI (bit-exact)."""
import numpy as np
import pytest

import oracle
from oracle import crt
from paper_2501_07047_gb300 import hefx, inputs

from hefx_testutil import empty_dev, to_dev, to_host

pytestmark = pytest.mark.gpu

PATHS = ["cudacore", "tensor"]


@pytest.fixture(scope="module")
def ctx():
    c = hefx.hefx_create(0)
    yield c
    hefx.hefx_destroy(c)


def convert(ctx, plan, a, Lp, path):
    B, L, n = a.shape
    din, dout = to_dev(a), empty_dev((B, Lp, n))
    hefx.hefx_basis_convert(ctx, plan, din, dout, B, path)
    return to_host(dout).reshape(B, Lp, n)


def available(ctx, plan, path, L, Lp, n):
    din, dout = empty_dev((1, L, n)), empty_dev((1, Lp, n))
    return hefx.raw_status("hefx_basis_convert", ctx, plan, din.data_ptr(), dout.data_ptr(), 0,
                           hefx.PATHS[path], 0) == hefx.HEFX_OK


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("logn,L,Lp,batch", [(0, 1, 1, 1), (3, 1, 3, 2), (5, 2, 2, 3), (7, 5, 3, 2),
                                             (10, 12, 28, 1), (9, 24, 8, 2), (12, 16, 40, 1), (6, 64, 64, 1),
                                             (11, 24, 56, 1)])
def test_bconv_matches_oracle(ctx, path, logn, L, Lp, batch):
    qs, ps = inputs.source_primes(L), inputs.special_primes(Lp)
    plan = hefx.hefx_bconv_plan_create(ctx, logn, qs, ps)
    try:
        n = 1 << logn
        if not available(ctx, plan, path, L, Lp, n):
            pytest.skip(f"{path} basis conversion not built for L={L}, L'={Lp}")
        a = inputs.residue_tensor(inputs.derive_seed(40, logn, L, Lp), batch, qs, n)
        got = convert(ctx, plan, a, Lp, path)
        assert (got == oracle.bconv(a, qs, ps)).all()
    finally:
        hefx.hefx_bconv_plan_destroy(plan)


@pytest.mark.parametrize("path", PATHS)
def test_bconv_config3_full_size(ctx, path):
    """16 x 24 limbs x 2^16 -> 8 limbs (the bench launch): every output of all 16 polynomials
    against the oracle, and 1024 sampled coefficients by big-integer CRT (the integer the fast
    conversion reduces), which pins the oracle itself at this size."""
    L, Lp, B, n = 24, 8, 16, 1 << 16
    qs, ps = inputs.source_primes(L), inputs.special_primes(Lp)
    plan = hefx.hefx_bconv_plan_create(ctx, 16, qs, ps)
    try:
        if not available(ctx, plan, path, L, Lp, n):
            pytest.skip("path not built")
        a = inputs.residue_tensor(inputs.derive_seed(3, 0), B, qs, n)
        got = convert(ctx, plan, a, Lp, path)
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=8) as ex:
            want = np.stack(list(ex.map(lambda b: oracle.bconv(a[b], qs, ps), range(B))))
        bad = np.argwhere(got != want)
        assert bad.size == 0, f"{len(bad)} outputs differ, first at {bad[0]}"
        rng = np.random.default_rng(9)
        for _ in range(1024):
            b, x = int(rng.integers(B)), int(rng.integers(n))
            y = crt.fast_conversion_integer([int(v) for v in a[b, :, x]], qs)
            assert [int(v) for v in want[b, :, x]] == [y % p for p in ps]
    finally:
        hefx.hefx_bconv_plan_destroy(plan)


@pytest.mark.parametrize("path", PATHS)
def test_bconv_edge_values(ctx, path):
    L, Lp, n = 6, 4, 256
    qs, ps = inputs.source_primes(L), inputs.special_primes(Lp)
    plan = hefx.hefx_bconv_plan_create(ctx, 8, qs, ps)
    try:
        if not available(ctx, plan, path, L, Lp, n):
            pytest.skip("path not built")
        a = np.zeros((3, L, n), np.uint32)
        for i, q in enumerate(qs):
            a[1, i] = q - 1
            a[2, i] = np.arange(n) % q
        got = convert(ctx, plan, a, Lp, path)
        assert (got[0] == 0).all()
        assert (got == oracle.bconv(a, qs, ps)).all()
    finally:
        hefx.hefx_bconv_plan_destroy(plan)


def test_bconv_validation(ctx):
    qs, ps = inputs.source_primes(3), inputs.special_primes(2)
    with pytest.raises(hefx.HefxError) as e:
        hefx.hefx_bconv_plan_create(ctx, 8, qs, [qs[0]])     # target repeats a source prime
    assert e.value.status == hefx.HEFX_EINVAL
    with pytest.raises(hefx.HefxError) as e:
        hefx.hefx_bconv_plan_create(ctx, 8, qs + [91], ps)   # 91 = 7 * 13
    assert e.value.status == hefx.HEFX_EINVAL
    plan = hefx.hefx_bconv_plan_create(ctx, 8, qs, ps)
    try:
        d = empty_dev(3 * 256 + 2 * 256)
        with pytest.raises(hefx.HefxError) as e:                 # overlapping buffers
            hefx.hefx_basis_convert(ctx, plan, d, d.data_ptr() + 16, 1, "cudacore")
        assert e.value.status == hefx.HEFX_EINVAL
    finally:
        hefx.hefx_bconv_plan_destroy(plan)


@pytest.mark.parametrize("logn,L,Lp,batch", [(4, 1, 2, 2), (8, 3, 4, 2), (10, 24, 8, 1), (16, 24, 8, 2)])
def test_bconv_exact_matches_oracle(ctx, logn, L, Lp, batch):
    qs, ps = inputs.source_primes(L), inputs.special_primes(Lp)
    plan = hefx.hefx_bconv_plan_create(ctx, logn, qs, ps)
    try:
        n = 1 << logn
        a = inputs.residue_tensor(inputs.derive_seed(48, logn, L, Lp), batch, qs, n)
        # the first coefficients hold small signed values, zero, +-Q/4 and values 2^-40 Q away
        # from +-Q/2 (outside the documented misrounding band of 2^-57 Q around Q/2)
        from math import prod
        Q = prod(qs)
        near = Q // 2 - (Q >> 40) if L > 1 else (Q - 1) // 2
        special = [0, 1, -1, 7, -7, 2 ** 45, -(2 ** 45), Q // 4, -(Q // 4), near, -near]
        for c, z in enumerate(special[:n]):
            for i, q in enumerate(qs):
                a[0, i, c] = z % q
        din, dout = to_dev(a), empty_dev((batch, Lp, n))
        hefx.hefx_basis_convert_exact(ctx, plan, din, dout, batch)
        got = to_host(dout).reshape(batch, Lp, n)
        cols = np.arange(n) if n <= 1024 else np.concatenate(
            [np.arange(len(special)), np.random.default_rng(2).choice(n, 200, replace=False)])
        for b in range(batch):
            want = np.array(crt.bconv_exact(a[b][:, cols].tolist(), qs, ps), dtype=np.uint32)
            bad = np.nonzero((got[b][:, cols] != want).any(axis=0))[0]
            assert bad.size == 0, f"batch {b}: columns {cols[bad][:8].tolist()} differ"
    finally:
        hefx.hefx_bconv_plan_destroy(plan)


def test_bconv_plan_rejects_accumulator_overflow(ctx):
    big = inputs.special_primes(40)
    st = hefx.raw_status("hefx_bconv_plan_create", ctx, 10, hefx._u32_array(big[:20]), 20,
                         hefx._u32_array(big[20:]), 20, hefx.ctypes.byref(hefx._vp()))
    assert st == hefx.HEFX_EUNSUPPORTED


@pytest.mark.parametrize("Lq,Lp", [(12, 28), (12, 36), (16, 40), (24, 56)])
def test_bconv_paper_shapes_tensor_path(ctx, Lq, Lp):
    """The paper's skewed conversion shapes at N = 2^16 run on the tensor path (up to 64 targets
    in one 256-column MMA) and match the oracle on every output; AUTO agrees."""
    qs, ps = inputs.source_primes(Lq), inputs.special_primes(Lp)
    n, B = 1 << 16, 2
    plan = hefx.hefx_bconv_plan_create(ctx, 16, qs, ps)
    try:
        assert available(ctx, plan, "tensor", Lq, Lp, n), "tensor path must be built for this shape"
        a = inputs.residue_tensor(inputs.derive_seed(41, Lq, Lp), B, qs, n)
        want = oracle.bconv(a, qs, ps)
        assert (convert(ctx, plan, a, Lp, "tensor") == want).all()
        assert (convert(ctx, plan, a, Lp, "auto") == want).all()
        hefx.hefx_bconv_check(ctx, plan)  # no bounded wait of the pipelined kernels expired
    finally:
        hefx.hefx_bconv_plan_destroy(plan)


@pytest.mark.parametrize("logn,L,Lp,batch", [(16, 48, 8, 2), (16, 24, 56, 2), (8, 48, 17, 3), (13, 1, 1, 5)])
def test_bconv_cudacore_tiled_shapes(ctx, logn, L, Lp, batch):
    """The CUDA-core conversion whose 256-coefficient tiles arrive by TMA (up to 48 sources):
    the most sources, several target chunks (step 1 kept in place between chunks), a single
    source; every output against the oracle, and no bounded wait expired."""
    qs, ps = inputs.source_primes(L), inputs.special_primes(Lp)
    n = 1 << logn
    plan = hefx.hefx_bconv_plan_create(ctx, logn, qs, ps)
    try:
        a = inputs.residue_tensor(inputs.derive_seed(42, logn, L, Lp), batch, qs, n)
        got = convert(ctx, plan, a, Lp, "cudacore")
        hefx.hefx_bconv_check(ctx, plan)
        assert (got == oracle.bconv(a, qs, ps)).all()
    finally:
        hefx.hefx_bconv_plan_destroy(plan)
