"""Serving loop on the GPU: every result is the same alone and in the mix (bit-exact), and
one request is checked stage by stage against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2501_07047_gb300 import hefx, inputs
from paper_2501_07047_gb300.serve import (GpuExecutor, N_SPECIAL, Request, poisson_requests, request_bytes, serve,
                                          serve_native)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = hefx.hefx_create(0)
    yield c
    hefx.hefx_destroy(c)


def oracle_request(ex, req):
    (a0, a1, b0, b1), (k0, k1) = ex.inputs_of(req)
    qs = ex.qprimes[:req.L]
    ps = ex.pprimes
    q = np.array(qs, dtype=np.uint64)[:, None]
    A0, A1, B0, B1 = (x.astype(np.uint64) for x in (a0, a1, b0, b1))
    d0 = (A0 * B0) % q
    d1 = ((A0 * B1) % q + (A1 * B0) % q) % q
    d2 = (A1 * B1) % q
    c = np.stack([oracle.intt(d2[i].astype(np.uint32), qs[i]) for i in range(req.L)])
    p = oracle.bconv(c, qs, ps)
    pn = np.stack([oracle.ntt(p[j], ps[j]) for j in range(N_SPECIAL)])
    ext = np.concatenate([d2, pn.astype(np.uint64)])
    mods = np.array(list(qs) + list(ps), dtype=np.uint64)[:, None]
    e0 = (ext * k0.astype(np.uint64)) % mods
    e1 = (ext * k1.astype(np.uint64)) % mods
    return [x.astype(np.uint32) for x in (d0, d1, e0, e1)]


@pytest.mark.parametrize("logn,L,variant", [(13, 8, 1), (16, 36, 0)])
def test_request_matches_oracle(ctx, logn, L, variant):
    """The smallest request shape and the largest one of the serving sweep (N = 2^16, L = 36),
    every output against the oracle composition."""
    ex = GpuExecutor(ctx, nstreams=2, seed=9)
    try:
        req = Request(0, logn, L, 0.0, variant=variant)
        st = serve([req], ex, keep_outputs=True)
        assert st["completed"] == 1
        for got, exp in zip(req.outputs, oracle_request(ex, req)):
            assert (got == exp).all()
    finally:
        ex.close()


def test_alone_equals_mix(ctx):
    ex = GpuExecutor(ctx, nstreams=8, seed=10)
    try:
        shapes = [(13, 8), (16, 36), (14, 20), (15, 11), (16, 9), (13, 30), (14, 8), (15, 36)]
        alone = []
        for k, (logn, L) in enumerate(shapes):
            r = Request(k, logn, L, 0.0, variant=k % 2)
            serve([r], ex, keep_outputs=True)
            alone.append(r.outputs)
        mix = [Request(k, logn, L, 0.0, variant=k % 2) for k, (logn, L) in enumerate(shapes)]
        st = serve(mix, ex, keep_outputs=True, max_slots=8)
        assert st["completed"] == len(shapes) and st["max_active"] >= 2
        for r, ref in zip(mix, alone):
            for got, exp in zip(r.outputs, ref):
                assert (got == exp).all(), (r.rid, r.logn, r.L)
    finally:
        ex.close()


def test_budget_limits_concurrency(ctx):
    ex = GpuExecutor(ctx, nstreams=4, seed=11)
    try:
        reqs = poisson_requests(12, 30, rate_hz=5000.0, logn_choices=(13, 14), lmin=8, lmax=12)
        for r in reqs:
            ex.warm(r.logn, r.L)
        budget = 2 * request_bytes(14, 12)
        st = serve(reqs, ex, budget_bytes=budget, max_slots=64)
        assert st["completed"] == 30 and st["memory_high_water_bytes"] <= budget
        big = Request(99, 16, 36, 0.0)
        st2 = serve([big], ex, budget_bytes=budget)
        assert big.status == "rejected" and st2["rejected"] == 1
    finally:
        ex.close()


def test_mult_plan_validation(ctx):
    """hefx_mult_plan_create refuses a conversion plan that does not map Q's primes to P's."""
    import torch
    logn, L = 10, 4
    qs, ps = inputs.source_primes(L), inputs.special_primes(N_SPECIAL)
    pq = hefx.hefx_params_create(ctx, logn, qs)
    pp = hefx.hefx_params_create(ctx, logn, ps)
    good = hefx.hefx_bconv_plan_create(ctx, logn, qs, ps)
    bad = hefx.hefx_bconv_plan_create(ctx, logn, inputs.source_primes(L + 1), ps)
    k = torch.zeros((L + N_SPECIAL, 1 << logn), dtype=torch.int32, device="cuda")
    try:
        with pytest.raises(hefx.HefxError) as e:
            hefx.hefx_mult_plan_create(ctx, pq, pp, bad, k, k, k, k)
        assert e.value.status == hefx.HEFX_EINVAL
        mp = hefx.hefx_mult_plan_create(ctx, pq, pp, good, k, k, k, k)
        buf = torch.zeros((4 * L, 1 << logn), dtype=torch.int32, device="cuda")
        # overlapping input and output buffers are refused before any launch
        assert hefx.raw_status("hefx_mult_front", ctx, mp, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 0) \
            == hefx.HEFX_EINVAL
        hefx.hefx_mult_plan_destroy(mp)
    finally:
        for pl in (good, bad):
            hefx.hefx_bconv_plan_destroy(pl)
        hefx.hefx_params_destroy(pq)
        hefx.hefx_params_destroy(pp)


def test_grouped_equals_alone_and_oracle(ctx):
    """Continuous batching across requests: requests admitted together run as groups of one
    ring degree in shared launches (hefx_mult_front_batch_host); every output equals the
    request served alone (bit for bit), and the small ones equal the oracle composition."""
    shapes = [(13, 8), (13, 30), (13, 12), (14, 20), (14, 9), (16, 36), (16, 8), (13, 36)]
    alone_ex = GpuExecutor(ctx, nstreams=2, seed=12)
    grouped_ex = GpuExecutor(ctx, nstreams=2, seed=12, grouped=True, max_group=4)
    try:
        alone = []
        for k, (logn, L) in enumerate(shapes):
            r = Request(k, logn, L, 0.0, variant=k % 2)
            serve([r], alone_ex, keep_outputs=True)
            alone.append(r.outputs)
        mix = [Request(k, logn, L, 0.0, variant=k % 2) for k, (logn, L) in enumerate(shapes)]
        st = serve(mix, grouped_ex, keep_outputs=True, max_slots=16)
        assert st["completed"] == len(shapes)
        for r, ref in zip(mix, alone):
            for got, exp in zip(r.outputs, ref):
                assert (got == exp).all(), (r.rid, r.logn, r.L)
        for r in mix:
            if r.logn == 13:
                for got, exp in zip(r.outputs, oracle_request(grouped_ex, r)):
                    assert (got == exp).all(), (r.rid, r.L)
    finally:
        alone_ex.close()
        grouped_ex.close()


def test_mult_batch_validation(ctx):
    """Batched requests must share the ring degree and P; the batch object bounds count and limbs."""
    import torch
    ex = GpuExecutor(ctx, nstreams=1, seed=13, slots=2)
    try:
        r13, r14 = ex.shape(13, 8), ex.shape(14, 8)
        mb = hefx.hefx_mult_batch_create(ctx, 2, 8)
        try:
            pl = ex.pool(13)["host_in"][0]
            slot = ex._slot()
            args = [pl[c] for c in range(4)]
            with pytest.raises(hefx.HefxError) as e:  # mixed ring degrees
                hefx.hefx_mult_front_batch_host(ctx, mb, [r13["mp"], r14["mp"]], *[[a, a] for a in args],
                                                [slot["h"], slot["h"]], [slot["d"], slot["d"]])
            assert e.value.status == hefx.HEFX_EINVAL
            with pytest.raises(hefx.HefxError) as e:  # more requests than the object holds
                hefx.hefx_mult_front_batch_host(ctx, mb, [r13["mp"]] * 3, *[[a] * 3 for a in args],
                                                [slot["h"]] * 3, [slot["d"]] * 3)
            assert e.value.status == hefx.HEFX_EINVAL
            big = ex.shape(13, 9)
            with pytest.raises(hefx.HefxError) as e:  # more limbs than the object holds
                hefx.hefx_mult_front_batch_host(ctx, mb, [big["mp"]], *[[a] for a in args], [slot["h"]], [slot["d"]])
            assert e.value.status == hefx.HEFX_EINVAL
            hefx.hefx_mult_front_batch_host(ctx, mb, [], [], [], [], [], [], [])  # nothing to do
            torch.cuda.synchronize()
        finally:
            hefx.hefx_mult_batch_destroy(mb)
    finally:
        ex.close()


@pytest.mark.parametrize("grouped", [False, True])
def test_resident_equals_host_and_oracle(ctx, grouped):
    """Resident serving (ciphertexts and results stay in device memory; hefx_mult_front_batch):
    every output equals the host-buffer path's (bit for bit), per request and in groups, and
    the small requests equal the oracle composition."""
    shapes = [(13, 8), (14, 20), (16, 36), (15, 11), (13, 30), (16, 9)]
    host_ex = GpuExecutor(ctx, nstreams=2, seed=13)
    res_ex = GpuExecutor(ctx, nstreams=2, seed=13, grouped=grouped, max_group=4, resident=True)
    try:
        ref = []
        for k, (logn, L) in enumerate(shapes):
            r = Request(k, logn, L, 0.0, variant=k % 2)
            serve([r], host_ex, keep_outputs=True)
            ref.append(r.outputs)
        mix = [Request(k, logn, L, 0.0, variant=k % 2) for k, (logn, L) in enumerate(shapes)]
        st = serve(mix, res_ex, keep_outputs=True, max_slots=8)
        assert st["completed"] == len(shapes)
        for r, exp_out in zip(mix, ref):
            for got, exp in zip(r.outputs, exp_out):
                assert (got == exp).all(), (r.rid, r.logn, r.L)
            if r.logn == 13:
                for got, exp in zip(r.outputs, oracle_request(res_ex, r)):
                    assert (got == exp).all(), (r.rid, r.L)
    finally:
        host_ex.close()
        res_ex.close()


def test_front_batch_validation(ctx):
    """hefx_mult_front_batch refuses an output that overlaps the request's inputs, before any
    launch."""
    import torch
    logn, L = 10, 4
    n = 1 << logn
    qs, ps = inputs.source_primes(L), inputs.special_primes(N_SPECIAL)
    pq = hefx.hefx_params_create(ctx, logn, qs)
    pp = hefx.hefx_params_create(ctx, logn, ps)
    bc = hefx.hefx_bconv_plan_create(ctx, logn, qs, ps)
    kq = torch.zeros((L, n), dtype=torch.int32, device="cuda")
    kp = torch.zeros((N_SPECIAL, n), dtype=torch.int32, device="cuda")
    mp = hefx.hefx_mult_plan_create(ctx, pq, pp, bc, kq, kq, kp, kp)
    mb = hefx.hefx_mult_batch_create(ctx, 2, L)
    try:
        ins = torch.zeros((4, L, n), dtype=torch.int32, device="cuda")
        out = torch.zeros(((4 * L + 2 * N_SPECIAL), n), dtype=torch.int32, device="cuda")
        work = torch.zeros(((2 * L + N_SPECIAL), n), dtype=torch.int32, device="cuda")
        hefx.hefx_mult_front_batch(ctx, mb, [mp], [ins[0]], [ins[1]], [ins[2]], [ins[3]], [out], [work])
        torch.cuda.synchronize()
        with pytest.raises(hefx.HefxError) as e:  # output over the inputs
            hefx.hefx_mult_front_batch(ctx, mb, [mp], [ins[0]], [ins[1]], [ins[2]], [ins[3]], [ins[0]], [work])
        assert e.value.status == hefx.HEFX_EINVAL
        with pytest.raises(hefx.HefxError) as e:  # more requests than the batch object holds
            hefx.hefx_mult_front_batch(ctx, mb, [mp] * 3, [ins[0]] * 3, [ins[1]] * 3, [ins[2]] * 3, [ins[3]] * 3,
                                       [out] * 3, [work] * 3)
        assert e.value.status == hefx.HEFX_EINVAL
    finally:
        hefx.hefx_mult_batch_destroy(mb)
        hefx.hefx_mult_plan_destroy(mp)
        hefx.hefx_bconv_plan_destroy(bc)
        hefx.hefx_params_destroy(pq)
        hefx.hefx_params_destroy(pp)


def test_native_loop_equals_python_and_oracle(ctx):
    """The native request loop (hefx_serve_run) on resident ciphertexts: every output equals the
    host-buffer path's, the small requests the oracle's; a Poisson run completes every request
    with several in flight inside the budget, and an oversize request is rejected."""
    shapes = [(13, 8), (14, 20), (16, 36), (15, 11), (13, 30), (16, 9), (14, 8), (13, 12)]
    host_ex = GpuExecutor(ctx, nstreams=2, seed=14)
    ex = GpuExecutor(ctx, nstreams=4, seed=14, grouped=True, max_group=4, resident=True)
    try:
        ref = []
        for k, (logn, L) in enumerate(shapes):
            r = Request(k, logn, L, 0.0, variant=k % 2)
            serve([r], host_ex, keep_outputs=True)
            ref.append(r.outputs)
        mix = [Request(k, logn, L, 0.0, variant=k % 2) for k, (logn, L) in enumerate(shapes)]
        st = serve_native(mix, ex, keep_outputs=True, max_slots=len(shapes))
        assert st["completed"] == len(shapes) and st["groups"] < len(shapes)  # some requests shared launches
        for r, exp_out in zip(mix, ref):
            for got, exp in zip(r.outputs, exp_out):
                assert (got == exp).all(), (r.rid, r.logn, r.L)
            if r.logn == 13:
                for got, exp in zip(r.outputs, oracle_request(ex, r)):
                    assert (got == exp).all(), (r.rid, r.L)
        reqs = poisson_requests(15, 80, rate_hz=20000.0, logn_choices=(13, 14), lmin=8, lmax=16)
        for r in reqs:
            ex.warm(r.logn, r.L)
        budget = 6 * request_bytes(14, 16)
        st = serve_native(reqs, ex, budget_bytes=budget, max_slots=16)
        assert st["completed"] == 80 and st["max_active"] >= 2 and st["memory_high_water_bytes"] <= budget
        big = Request(99, 16, 36, 0.0)
        ex.warm(16, 36)
        st = serve_native([big], ex, budget_bytes=budget)
        assert big.status == "rejected" and st["rejected"] == 1
    finally:
        host_ex.close()
        ex.close()

