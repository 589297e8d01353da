"""Host-resident transforms with overlapped copies (hostio.NttRoundTrip): chunks of a pinned
batch round-trip bit for bit, the forward-only form equals the oracle, and the buffer
rotation stays correct across calls and a ragged last chunk."""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_07047_gb300 import hefx, inputs
from paper_2501_07047_gb300.hostio import NttRoundTrip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = hefx.hefx_create(0)
    yield c
    hefx.hefx_destroy(c)


@pytest.mark.parametrize("logn,L,batch,chunk", [(12, 3, 5, 2), (16, 4, 4, 1)])
def test_round_trip_and_forward(ctx, logn, L, batch, chunk):
    n = 1 << logn
    primes = inputs.source_primes(L)
    p = hefx.hefx_params_create(ctx, logn, primes)
    try:
        x = inputs.residue_tensor(inputs.derive_seed(90, logn), batch, primes, n)
        h_in = torch.from_numpy(x.view(np.int32).copy()).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        rt = NttRoundTrip(ctx, p, L, n, chunk=chunk)
        for _ in range(3):  # rotation across calls
            h_out.zero_()
            rt.run(h_in, h_out)
            rt.join()
            torch.cuda.synchronize()
            assert torch.equal(h_out, h_in)
        fw = NttRoundTrip(ctx, p, L, n, chunk=chunk, ops=("fwd",))
        fw.run(h_in, h_out)
        fw.join()
        torch.cuda.synchronize()
        assert (h_out.numpy().view(np.uint32) == oracle.ntt_batch(x, primes)).all()
    finally:
        hefx.hefx_params_destroy(p)
