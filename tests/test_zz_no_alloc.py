"""hefx_poly_mul_noalloc: the tensor-path product with its workspace in a fixed array inside
the library, for callers that cannot allocate device memory while running (a memory plan
fixed up front, or a loop where a cudaMalloc could stall on device-wide synchronization).
Checked through the C ABI against hefx_poly_mul (tensor path) and against the oracle on two
calls in a row, and in its aliasing forms (a == b, c == b); results are integers, so the
tolerance is exact equality.  Kept in its own file, collected last."""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_07047_gb300 import hefx, inputs

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32).copy()).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint32)


def test_noalloc_matches_poly_mul_twice():
    ctx = hefx.hefx_create(0)
    primes = inputs.source_primes(3)
    p = hefx.hefx_params_create(ctx, 16, primes)
    try:
        shape = (2, 3, 1 << 16)  # 2 * 3 * 2^16 residues, inside the 2^21-residue array
        refs, outs = [], []
        for call in range(2):
            a = inputs.residue_tensor(inputs.derive_seed(77, call, 0), 2, primes, 1 << 16)
            b = inputs.residue_tensor(inputs.derive_seed(77, call, 1), 2, primes, 1 << 16)
            da, db = dev(a), dev(b)
            ref = torch.empty(shape, dtype=torch.int32, device="cuda")
            hefx.hefx_poly_mul(ctx, p, da, db, ref, 2, "tensor")  # also builds the tensor tables
            hefx.hefx_stream_check(ctx, p)
            got = torch.full(shape, -1, dtype=torch.int32, device="cuda")
            hefx.hefx_poly_mul_noalloc(ctx, p, da, db, got, 2)
            hefx.hefx_stream_check(ctx, p)
            refs.append(host(ref))
            outs.append(host(got))
            assert (outs[-1] == oracle.polymul_batch(a, b, primes)).all()
        for r, g in zip(refs, outs):
            assert (g == r).all()
        assert not (refs[0] == refs[1]).all()  # the two calls really computed different products
        big = torch.empty((12, 3, 1 << 16), dtype=torch.int32, device="cuda")  # 12*3*2^16 > 2^21
        with pytest.raises(hefx.HefxError) as e:
            hefx.hefx_poly_mul_noalloc(ctx, p, big, big, big, 12)
        assert e.value.status == hefx.HEFX_EINVAL
    finally:
        hefx.hefx_params_destroy(p)
        hefx.hefx_destroy(ctx)


def test_noalloc_aliasing_forms():
    """a == b (the square, whose forward transform goes through the static array) and the
    in-place forms c == b and c == a == b, each bit-exact against hefx_poly_mul."""
    ctx = hefx.hefx_create(0)
    primes = inputs.source_primes(2)
    p = hefx.hefx_params_create(ctx, 14, primes)
    try:
        shape = (3, 2, 1 << 14)
        a = inputs.residue_tensor(inputs.derive_seed(78, 0), 3, primes, 1 << 14)
        b = inputs.residue_tensor(inputs.derive_seed(78, 1), 3, primes, 1 << 14)
        da, db = dev(a), dev(b)
        sq_ref = torch.empty(shape, dtype=torch.int32, device="cuda")
        hefx.hefx_poly_mul(ctx, p, da, da, sq_ref, 3, "tensor")
        hefx.hefx_stream_check(ctx, p)
        sq = torch.full(shape, -1, dtype=torch.int32, device="cuda")
        hefx.hefx_poly_mul_noalloc(ctx, p, da, da, sq, 3)
        hefx.hefx_stream_check(ctx, p)
        assert (host(sq) == host(sq_ref)).all()
        assert (host(sq).reshape(shape) == oracle.polymul_batch(a, a, primes)).all()
        ab_ref = torch.empty(shape, dtype=torch.int32, device="cuda")
        hefx.hefx_poly_mul(ctx, p, da, db, ab_ref, 3, "tensor")
        db2 = dev(b)
        hefx.hefx_poly_mul_noalloc(ctx, p, da, db2, db2, 3)  # c == b
        hefx.hefx_stream_check(ctx, p)
        assert (host(db2) == host(ab_ref)).all()
        assert (host(da) == a).all()  # a untouched
        da2 = dev(a)
        hefx.hefx_poly_mul_noalloc(ctx, p, da2, da2, da2, 3)  # c == a == b
        hefx.hefx_stream_check(ctx, p)
        assert (host(da2) == host(sq_ref)).all()
    finally:
        hefx.hefx_params_destroy(p)
        hefx.hefx_destroy(ctx)
