"""The modular-reduction ablation (Sec. V-F): every twiddle-product reduction of the
CUDA-core NTT (Shoup, Montgomery, Barrett) and every VecModMul reduction (Montgomery,
Barrett, BAT lazy on the tensor cores) return the oracle's results bit for bit; unsupported
combinations are refused."""
import numpy as np
import pytest

import oracle
from paper_2501_07047_gb300 import hefx, inputs

from hefx_testutil import empty_dev, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = hefx.hefx_create(0)
    yield c
    hefx.hefx_destroy(c)


@pytest.mark.parametrize("red", ["shoup", "montgomery", "barrett"])
@pytest.mark.parametrize("bits", [28, 30])
def test_ntt_reductions_match_oracle(ctx, red, bits):
    n, L, batch = 1 << 16, 3, 2
    primes = inputs.ntt_primes(L, bits)
    p = hefx.hefx_params_create(ctx, 16, primes)
    try:
        hefx.hefx_params_set_reduction(ctx, p, red, "montgomery")
        a = inputs.residue_tensor(inputs.derive_seed(80, bits), batch, primes, n)
        d = to_dev(a)
        hefx.hefx_ntt_fwd(ctx, p, d, batch, "cudacore")
        got = to_host(d).reshape(a.shape)
        assert (got == oracle.ntt_batch(a, primes)).all()
        hefx.hefx_ntt_inv(ctx, p, d, batch, "cudacore")
        assert (to_host(d).reshape(a.shape) == a).all()
    finally:
        hefx.hefx_params_destroy(p)


@pytest.mark.parametrize("red", ["montgomery", "barrett", "bat_lazy"])
def test_vec_mod_mul_reductions(ctx, red):
    n, L = 1 << 12, 4
    primes = list(inputs.source_primes(2)) + list(inputs.special_primes(2))
    p = hefx.hefx_params_create(ctx, 12, primes)
    try:
        hefx.hefx_params_set_reduction(ctx, p, "shoup", red)
        x = inputs.residue_tensor(inputs.derive_seed(81, 0), 1, primes, n)
        y = inputs.residue_tensor(inputs.derive_seed(81, 1), 1, primes, n)
        # extremes: q - 1 times q - 1, zero
        x[0, :, 0] = [q - 1 for q in primes]
        y[0, :, 0] = [q - 1 for q in primes]
        x[0, :, 1] = 0
        dx, dy, dz = to_dev(x), to_dev(y), empty_dev(x.shape)
        hefx.hefx_vec_mod_mul(ctx, p, dx, dy, dz, 1)
        q = np.asarray(primes, dtype=np.uint64)[:, None]
        want = ((x[0].astype(np.uint64) * y[0]) % q).astype(np.uint32)
        assert (to_host(dz).reshape(x.shape)[0] == want).all()
    finally:
        hefx.hefx_params_destroy(p)


@pytest.mark.parametrize("logn,L,batch", [(16, 24, 1), (9, 3, 5), (10, 7, 3)])
def test_vec_mod_mul_bat_lazy_sizes(ctx, logn, L, batch):
    """BAT lazy reduction (tensor cores) over many 512-element steps, limb changes inside a
    CTA's steps and 30-bit primes; extremes q - 1 and 0."""
    n = 1 << logn
    primes = list(inputs.source_primes(L - L // 2)) + list(inputs.special_primes(L // 2))
    p = hefx.hefx_params_create(ctx, logn, primes)
    try:
        hefx.hefx_params_set_reduction(ctx, p, "shoup", "bat_lazy")
        x = inputs.residue_tensor(inputs.derive_seed(82, logn), batch, primes, n)
        y = inputs.residue_tensor(inputs.derive_seed(83, logn), batch, primes, n)
        q = np.asarray(primes, dtype=np.uint64)[None, :, None]
        x[:, :, :3] = (q - 1).astype(np.uint32)
        y[:, :, :2] = (q - 1).astype(np.uint32)
        y[:, :, 2] = 0
        dx, dy, dz = to_dev(x), to_dev(y), empty_dev(x.shape)
        hefx.hefx_vec_mod_mul(ctx, p, dx, dy, dz, batch)
        want = ((x.astype(np.uint64) * y) % q).astype(np.uint32)
        assert (to_host(dz).reshape(x.shape) == want).all()
        hefx.hefx_stream_check(ctx, p)  # no MMA wait ran out
    finally:
        hefx.hefx_params_destroy(p)


def test_reduction_refusals(ctx):
    p12 = hefx.hefx_params_create(ctx, 12, inputs.source_primes(1))
    p16 = hefx.hefx_params_create(ctx, 16, inputs.source_primes(1))
    try:
        d = empty_dev((1, 1, 1 << 16))
        assert hefx.raw_status("hefx_params_set_reduction", p16, 0, 0) == hefx.HEFX_EINVAL  # Shoup VecModMul
        assert hefx.raw_status("hefx_params_set_reduction", p16, 7, 1) == hefx.HEFX_EINVAL
        p8 = hefx.hefx_params_create(ctx, 8, inputs.source_primes(1))
        try:  # the BAT lazy kernel takes 512-element steps inside one limb
            assert hefx.raw_status("hefx_params_set_reduction", p8, 0, 3) == hefx.HEFX_EUNSUPPORTED
        finally:
            hefx.hefx_params_destroy(p8)
        hefx.hefx_params_set_reduction(ctx, p12, "barrett", "montgomery")
        assert hefx.raw_status("hefx_ntt_fwd", ctx, p12, d.data_ptr(), 1, hefx.PATHS["cudacore"], 0) \
            == hefx.HEFX_EUNSUPPORTED
        hefx.hefx_params_set_reduction(ctx, p16, "montgomery", "montgomery")
        assert hefx.raw_status("hefx_poly_mul", ctx, p16, d.data_ptr(), d.data_ptr(), d.data_ptr(), 1,
                               hefx.PATHS["cudacore"], 0) == hefx.HEFX_EUNSUPPORTED
        # back to the default: everything works again
        hefx.hefx_params_set_reduction(ctx, p16, "shoup", "montgomery")
        assert hefx.raw_status("hefx_poly_mul", ctx, p16, d.data_ptr(), d.data_ptr(), d.data_ptr(), 1,
                               hefx.PATHS["cudacore"], 0) == hefx.HEFX_OK
    finally:
        hefx.hefx_params_destroy(p12)
        hefx.hefx_params_destroy(p16)
