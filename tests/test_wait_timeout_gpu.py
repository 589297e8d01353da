"""Failure detection without a fault: the bounded device wait that every tcgen05 / TMA
pipeline of the library uses runs out on an mbarrier that nothing arrives on, the kernel
frees its TMEM and returns, hefx_stream_check reports HEFX_ETIMEOUT, and the next calls on the
same context are bit-exact against the oracle."""
import pytest

import oracle
from paper_2501_07047_gb300 import hefx, inputs

from hefx_testutil import to_dev, to_host

pytestmark = pytest.mark.gpu


def test_wait_runs_out_and_context_stays_usable():
    import torch
    assert torch.cuda.is_available()
    ctx = hefx.hefx_create(0)
    primes = inputs.source_primes(2)
    p = hefx.hefx_params_create(ctx, 16, primes)
    try:
        hefx.hefx_wait_check(ctx, p, 2_000_000_000, arrive=True)   # the barrier completes
        hefx.hefx_stream_check(ctx, p)
        hefx.hefx_wait_check(ctx, p, 1_000_000, arrive=False)      # nothing arrives: 1 ms, then give up
        with pytest.raises(hefx.HefxError) as e:
            hefx.hefx_stream_check(ctx, p)
        assert e.value.status == hefx.HEFX_ETIMEOUT
        hefx.hefx_stream_check(ctx, p)                              # the flag was read and cleared
        with pytest.raises(hefx.HefxError) as e:
            hefx.hefx_wait_check(ctx, p, 3_000_000_000, arrive=False)
        assert e.value.status == hefx.HEFX_EINVAL
        data = inputs.residue_tensor(inputs.derive_seed(90, 0), 2, primes, 1 << 16)
        want = oracle.ntt_batch(data, primes)
        for path in ("tensor", "cudacore"):
            d = to_dev(data)
            hefx.hefx_ntt_fwd(ctx, p, d, 2, path)
            hefx.hefx_stream_check(ctx, p)
            assert (to_host(d).reshape(data.shape) == want).all(), path
    finally:
        hefx.hefx_params_destroy(p)
        hefx.hefx_destroy(ctx)
