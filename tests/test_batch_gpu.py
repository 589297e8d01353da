"""GPU parity of batched uneven polynomial products (one graph launch) against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_07047_gb300 import hefx, inputs
from paper_2501_07047_gb300.batch import UnevenBatch

from hefx_testutil import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = hefx.hefx_create(0)
    yield c
    hefx.hefx_destroy(c)


def expect(batch, j):
    logn, L = batch.shapes[j]
    a, b = batch.host_inputs(j)
    return oracle.polymul_batch(a[None], b[None], batch.primes[:L])[0]


def test_small_mix_graph_replay(ctx):
    shapes = [(3, 1), (6, 2), (10, 3), (12, 5), (13, 2), (14, 1), (15, 2), (16, 3), (12, 1), (16, 1), (4, 4), (11, 2)]
    batch = UnevenBatch(ctx, shapes, seed=41, lmax=8)
    try:
        s = torch.cuda.Stream()
        for rep in range(3):  # first call captures the graph, the others replay it
            for c in batch.c:
                c.zero_()
            with torch.cuda.stream(s):
                batch.run(s)
            s.synchronize()
            for j in range(len(shapes)):
                assert (batch.c[j].cpu().numpy().view(np.uint32) == expect(batch, j)).all(), (rep, j, shapes[j])
    finally:
        batch.close()


def test_aliasing_and_default_stream(ctx):
    primes = inputs.source_primes(4)
    p12 = hefx.hefx_params_create(ctx, 12, primes)
    p16 = hefx.hefx_params_create(ctx, 16, primes)
    try:
        ha = inputs.residue_tensor(5, 1, primes[:3], 4096)[0]
        hb = inputs.residue_tensor(6, 1, primes[:3], 4096)[0]
        ga = inputs.residue_tensor(7, 1, primes[:2], 65536)[0]
        a1, b1 = to_dev(ha), to_dev(hb)          # c aliases a
        a2, b2 = to_dev(ha), to_dev(hb)          # c aliases b
        a3 = to_dev(ga)                          # a == b == c (square in place)
        a4, c4 = to_dev(ga), torch.empty((2, 65536), dtype=torch.int32, device="cuda")  # a == b
        jobs = [(p12, 3, a1, b1, a1), (p12, 3, a2, b2, b2), (p16, 2, a3, a3, a3), (p16, 2, a4, a4, c4)]
        plan = hefx.hefx_batch_plan_create(ctx, jobs)
        try:
            hefx.hefx_batch_polymul(ctx, plan, None)  # legacy stream: direct launches
            ab = oracle.polymul_batch(ha[None], hb[None], primes[:3])[0]
            sq = oracle.polymul_batch(ga[None], ga[None], primes[:2])[0]
            assert (to_host(a1).reshape(ab.shape) == ab).all()
            assert (to_host(b2).reshape(ab.shape) == ab).all()
            assert (to_host(a3).reshape(sq.shape) == sq).all()
            assert (to_host(c4).reshape(sq.shape) == sq).all()
        finally:
            hefx.hefx_batch_plan_destroy(plan)
        with pytest.raises(hefx.HefxError) as e:
            hefx.hefx_batch_plan_create(ctx, [(p12, 5, a1, b1, a1)])  # more limbs than the params hold
        assert e.value.status == hefx.HEFX_EINVAL
        with pytest.raises(hefx.HefxError) as e:
            hefx.hefx_batch_plan_create(ctx, [(p12, 1, a1, b1, a1)], "tensor")
        assert e.value.status == hefx.HEFX_EUNSUPPORTED
    finally:
        hefx.hefx_params_destroy(p12)
        hefx.hefx_params_destroy(p16)


def test_config4_full_size(ctx):
    """256 jobs, N uniform in {2^12..2^16}, L uniform in [4, 32] (the bench batch): every limb
    of every job against the oracle after a graph replay."""
    from concurrent.futures import ThreadPoolExecutor
    shapes = inputs.uneven_jobs(inputs.derive_seed(4), 256)
    batch = UnevenBatch(ctx, shapes, seed=4)
    try:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            batch.run(s)
            batch.run(s)  # replay: same inputs, same outputs
        s.synchronize()
        ins = [batch.host_inputs(j) for j in range(len(shapes))]

        def want_of(j):
            a, b = ins[j]
            return oracle.polymul_batch(a[None], b[None], batch.primes[:shapes[j][1]])[0]

        with ThreadPoolExecutor(max_workers=8) as ex:
            wants = list(ex.map(want_of, range(len(shapes))))
        for j, want in enumerate(wants):
            got = batch.c[j].cpu().numpy().view(np.uint32)
            assert (got == want).all(), (j, shapes[j])
    finally:
        batch.close()


def test_fused_batch_edges(ctx):
    """The one-launch batch with every ring degree it takes (2^10 .. 2^16), squares, c aliasing
    a or b, and counts of split rows (2^14 .. 2^16) that leave the last cluster task partly
    filled (scratch rows fill it); one launch, every limb against the oracle, replayed."""
    primes = inputs.source_primes(5)
    params = {logn: hefx.hefx_params_create(ctx, logn, primes) for logn in range(10, 17)}
    try:
        jobs, expect_list, keep = [], [], []
        spec = [(10, 3, "ab"), (11, 2, "sq"), (12, 5, "ca"), (13, 1, "cb"), (14, 3, "ab"), (14, 1, "sq"),
                (15, 1, "ab"), (15, 2, "sq"), (16, 3, "cb"), (16, 2, "ab"), (13, 4, "sq"), (12, 1, "ab")]
        for k, (logn, L, kind) in enumerate(spec):
            n = 1 << logn
            ha = inputs.residue_tensor(inputs.derive_seed(120, k, 0), 1, primes[:L], n)[0]
            hb = inputs.residue_tensor(inputs.derive_seed(120, k, 1), 1, primes[:L], n)[0]
            a, b = to_dev(ha), to_dev(hb)
            if kind == "sq":
                c = torch.empty((L, n), dtype=torch.int32, device="cuda")
                jobs.append((params[logn], L, a, a, c))
                want = oracle.polymul_batch(ha[None], ha[None], primes[:L])[0]
            elif kind == "ca":
                c = a
                jobs.append((params[logn], L, a, b, c))
                want = oracle.polymul_batch(ha[None], hb[None], primes[:L])[0]
            elif kind == "cb":
                c = b
                jobs.append((params[logn], L, a, b, c))
                want = oracle.polymul_batch(ha[None], hb[None], primes[:L])[0]
            else:
                c = torch.empty((L, n), dtype=torch.int32, device="cuda")
                jobs.append((params[logn], L, a, b, c))
                want = oracle.polymul_batch(ha[None], hb[None], primes[:L])[0]
            keep.append((a, b, c))
            expect_list.append((c, want))
        plan = hefx.hefx_batch_plan_create(ctx, jobs)
        try:
            assert hefx.hefx_batch_plan_launches(plan) == 1
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                hefx.hefx_batch_polymul(ctx, plan, s)
            s.synchronize()
            for k, (c, want) in enumerate(expect_list):
                assert (to_host(c).reshape(want.shape) == want).all(), spec[k]
        finally:
            hefx.hefx_batch_plan_destroy(plan)
        # a ring degree below 2^10 keeps the per-size-class launches
        p8 = hefx.hefx_params_create(ctx, 8, primes)
        try:
            ha = inputs.residue_tensor(inputs.derive_seed(121, 0), 1, primes[:2], 256)[0]
            a, c = to_dev(ha), torch.empty((2, 256), dtype=torch.int32, device="cuda")
            plan = hefx.hefx_batch_plan_create(ctx, [(p8, 2, a, a, c), (params[12], 1, keep[0][0], keep[0][0],
                                                                          torch.empty((1, 4096), dtype=torch.int32,
                                                                                      device="cuda"))])
            try:
                assert hefx.hefx_batch_plan_launches(plan) > 1
                hefx.hefx_batch_polymul(ctx, plan, None)
                assert (to_host(c).reshape(2, 256) == oracle.polymul_batch(ha[None], ha[None], primes[:2])[0]).all()
            finally:
                hefx.hefx_batch_plan_destroy(plan)
        finally:
            hefx.hefx_params_destroy(p8)
    finally:
        for p in params.values():
            hefx.hefx_params_destroy(p)
