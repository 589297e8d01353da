"""GPU parity of the key-switching pieces (VecModAdd, key inner product, ModDown, Rescale) and
of the composed HE-Mult against the oracle, bit for bit, plus the decryption relation of a
genuine switching key on the GPU's result."""
import numpy as np
import pytest

import oracle
from oracle import keyswitch as oks
from paper_2501_07047_gb300 import hefx, inputs

from hefx_testutil import to_dev as dev, to_host as host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hx():
    ctx = hefx.hefx_create(0)
    yield hefx, ctx
    hefx.hefx_destroy(ctx)


def _res(seed, rows, primes, n):
    return inputs.residue_tensor(inputs.derive_seed(*seed), rows, primes, n)


@pytest.mark.parametrize("logn,L,K", [(8, 3, 2), (12, 6, 4), (16, 24, 8)])
def test_mod_down(hx, logn, L, K):
    hefx, ctx = hx
    n, batch = 1 << logn, 2
    qs, ps = inputs.source_primes(L), inputs.special_primes(K)
    x = np.stack([_res((60, logn, b), 1, list(qs) + list(ps), n)[0] for b in range(batch)])
    plan = hefx.hefx_bconv_plan_create(ctx, logn, ps, qs)
    dx, dout = dev(x), dev(np.zeros((batch, L, n), dtype=np.uint32))
    hefx.hefx_mod_down(ctx, plan, dx, dout, batch)
    got = host(dout)
    if logn <= 12:
        assert np.array_equal(got, oracle.moddown(x, qs, ps))
    else:  # full size: every limb of sampled coefficients
        cols = np.random.default_rng(1).choice(n, 256, replace=False)
        want = oracle.moddown(x[:, :, cols], qs, ps)
        assert np.array_equal(got[:, :, cols], want)
    hefx.hefx_bconv_plan_destroy(plan)


@pytest.mark.parametrize("logn,L,K,alpha,batch", [(8, 5, 2, 2, 1), (12, 6, 3, 3, 2), (10, 7, 1, 7, 1),
                                                    (16, 48, 16, 16, 1), (16, 24, 8, 8, 2)])
def test_mod_up(hx, logn, L, K, alpha, batch):
    """One-launch ModUp of every digit (ragged last digit, single digit, batch 2) equals the
    oracle's per-digit conversions and copies."""
    hefx, ctx = hx
    n = 1 << logn
    qs, ps = inputs.source_primes(L), inputs.special_primes(K)
    c = np.stack([_res((67, logn, b), 1, qs, n)[0] for b in range(batch)])
    c[:, :, 0] = np.asarray(qs, dtype=np.uint32)[None, :] - 1  # extremes
    c[:, :, 1] = 0
    plan = hefx.hefx_modup_plan_create(ctx, logn, qs, ps, alpha)
    dnum = hefx.hefx_modup_plan_dnum(plan)
    assert dnum == len(oks.digit_ranges(L, alpha))
    dc = dev(c)
    dU = dev(np.full((batch, dnum, L + K, n), 0xFFFFFFFF, dtype=np.uint32))
    hefx.hefx_mod_up(ctx, plan, dc, dU, batch)
    got = host(dU)
    cols = np.arange(n) if logn <= 12 else np.sort(np.random.default_rng(2).choice(n, 512, replace=False))
    for b in range(batch):
        want = oks.modup(c[b][:, cols], qs, ps, alpha)
        assert np.array_equal(got[b][:, :, cols], want)
    hefx.hefx_modup_plan_destroy(plan)


def test_mod_up_errors(hx):
    hefx, ctx = hx
    qs, ps = inputs.source_primes(4), inputs.special_primes(2)
    with pytest.raises(hefx.HefxError):
        hefx.hefx_modup_plan_create(ctx, 8, qs, ps, 0)  # alpha outside [1, L]
    with pytest.raises(hefx.HefxError):
        hefx.hefx_modup_plan_create(ctx, 8, qs, ps, 5)
    with pytest.raises(hefx.HefxError):
        hefx.hefx_modup_plan_create(ctx, 8, qs, list(ps[:1]) + [qs[0]], 2)  # repeated prime
    plan = hefx.hefx_modup_plan_create(ctx, 8, qs, ps, 2)
    buf = dev(np.zeros((2 * 6 + 4, 256), dtype=np.uint32))
    # d_U overlapping d_c
    assert hefx.raw_status("hefx_mod_up", ctx, plan, buf.data_ptr(), buf.data_ptr() + 1024, 1, 0) == hefx.HEFX_EINVAL
    assert hefx.raw_status("hefx_mod_up", ctx, 0, buf.data_ptr(), buf.data_ptr(), 1, 0) == hefx.HEFX_EINVAL
    hefx.hefx_modup_plan_destroy(plan)


@pytest.mark.parametrize("logn,L", [(6, 2), (10, 5), (16, 24)])
def test_rescale(hx, logn, L):
    hefx, ctx = hx
    n = 1 << logn
    qs = inputs.source_primes(L)
    p = hefx.hefx_params_create(ctx, logn, qs)
    x = np.stack([_res((61, logn, b), 1, qs, n)[0] for b in range(2)])
    dx, dout = dev(x), dev(np.zeros((2, L - 1, n), dtype=np.uint32))
    hefx.hefx_rescale(ctx, p, dx, dout, 2)
    assert np.array_equal(host(dout), oracle.rescale(x, qs))
    # in place with batch 1: the result occupies the first L - 1 rows
    d1 = dev(x[0])
    hefx.hefx_rescale(ctx, p, d1, d1, 1)
    assert np.array_equal(host(d1)[:L - 1], oracle.rescale(x[0], qs))
    hefx.hefx_params_destroy(p)


@pytest.mark.parametrize("logn,L,batch", [(10, 5, 2), (14, 6, 2), (15, 9, 1), (16, 24, 2), (16, 48, 2), (17, 4, 1)])
def test_rescale_ntt(hx, logn, L, batch):
    """NTT(Rescale(x)) over q_0..q_{L-2}: fused on the forward transform's load for N >= 2^14,
    two steps below; equal to the oracle's rescale followed by its forward NTT."""
    hefx, ctx = hx
    n = 1 << logn
    qs = inputs.source_primes(L) if logn <= 16 else inputs.ntt_primes(L, 28, 2 << logn)
    p = hefx.hefx_params_create(ctx, logn, qs)
    x = np.stack([_res((68, logn, b), 1, qs, n)[0] for b in range(batch)])
    x[:, :, 0] = np.asarray(qs, dtype=np.uint32)[None, :] - 1  # extremes, last limb included
    x[:, :, 1] = 0
    dx, dout = dev(x), dev(np.zeros((batch, L - 1, n), dtype=np.uint32))
    hefx.hefx_rescale_ntt(ctx, p, dx, dout, batch)
    want = oracle.ntt_batch(oracle.rescale(x, qs), list(qs[:-1]))
    assert np.array_equal(host(dout), want)
    assert np.array_equal(host(dx), x)  # input untouched
    hefx.hefx_params_destroy(p)


@pytest.mark.parametrize("logn,nl,dnum,batch", [(8, 5, 3, 1), (12, 10, 1, 2), (16, 32, 3, 1)])
def test_key_inner_product_and_add(hx, logn, nl, dnum, batch):
    hefx, ctx = hx
    n = 1 << logn
    qs = list(inputs.source_primes(nl - nl // 3)) + list(inputs.special_primes(nl // 3))
    p = hefx.hefx_params_create(ctx, logn, qs)
    dig = np.stack([np.stack([_res((62, logn, b, j), 1, qs, n)[0] for j in range(dnum)]) for b in range(batch)])
    evk = np.stack([np.stack([_res((63, logn, j, k), 1, qs, n)[0] for k in range(2)]) for j in range(dnum)])
    dd, de, do = dev(dig), dev(evk), dev(np.zeros((batch, 2, nl, n), dtype=np.uint32))
    hefx.hefx_key_inner_product(ctx, p, dd, de, do, dnum, batch)
    got = host(do)
    for b in range(batch):
        assert np.array_equal(got[b], oracle.key_inner_product(dig[b], evk, qs))
    # VecModAdd on the two halves, in place into the first
    hefx.hefx_vec_mod_add(ctx, p, do[0, 0], do[0, 1], do[0, 0], 1)
    q = np.asarray(qs, dtype=np.uint64)[:, None]
    want = ((got[0, 0].astype(np.uint64) + got[0, 1]) % q).astype(np.uint32)
    assert np.array_equal(host(do)[0, 0], want)
    hefx.hefx_params_destroy(p)


@pytest.mark.parametrize("logn,L,batch", [(8, 3, 2), (16, 24, 1)])
def test_ntt_inv_hadamard(hx, logn, L, batch):
    """INTT(x o y) equals the oracle's product followed by its inverse NTT; a null d2 leaves
    the tensor product's other outputs unchanged."""
    hefx, ctx = hx
    n = 1 << logn
    qs = inputs.source_primes(L)
    p = hefx.hefx_params_create(ctx, logn, qs)
    x = np.stack([_res((69, logn, b), 1, qs, n)[0] for b in range(batch)])
    y = np.stack([_res((70, logn, b), 1, qs, n)[0] for b in range(batch)])
    q = np.asarray(qs, dtype=np.uint64)[None, :, None]
    dx, dy, dout = dev(x), dev(y), dev(np.zeros_like(x))
    hefx.hefx_ntt_inv_hadamard(ctx, p, dx, dy, dout, batch)
    want = oracle.ntt_batch(((x.astype(np.uint64) * y) % q).astype(np.uint32), qs, inverse=True)
    assert np.array_equal(host(dout), want)
    assert hefx.raw_status("hefx_ntt_inv_hadamard", ctx, p, dx.data_ptr(), dy.data_ptr(), dx.data_ptr(), batch, 0) \
        == hefx.HEFX_EINVAL  # in place on an input
    d0, d1 = dev(np.zeros_like(x)), dev(np.zeros_like(x))
    hefx.hefx_tensor_product(ctx, p, dx, dx, dy, dy, d0, d1, None, batch)
    assert np.array_equal(host(d0), ((x.astype(np.uint64) * y) % q).astype(np.uint32))
    hefx.hefx_params_destroy(p)


def test_keyswitch_errors(hx):
    hefx, ctx = hx
    q1 = inputs.source_primes(1)
    p1 = hefx.hefx_params_create(ctx, 8, q1)
    buf = dev(np.zeros((8, 256), dtype=np.uint32))  # every range named below lies inside it
    assert hefx.raw_status("hefx_rescale", ctx, p1, buf.data_ptr(), buf.data_ptr(), 1, 0) == hefx.HEFX_EINVAL
    assert hefx.raw_status("hefx_rescale_ntt", ctx, p1, buf.data_ptr(), buf.data_ptr() + 2048, 1, 0) \
        == hefx.HEFX_EINVAL  # one limb: nothing to rescale
    p3 = hefx.hefx_params_create(ctx, 8, inputs.source_primes(3))
    # rescaled output overlapping the input
    assert hefx.raw_status("hefx_rescale_ntt", ctx, p3, buf.data_ptr(), buf.data_ptr() + 1024, 1, 0) \
        == hefx.HEFX_EINVAL
    hefx.hefx_params_set_reduction(ctx, p3, "barrett", "montgomery")
    assert hefx.raw_status("hefx_rescale_ntt", ctx, p3, buf.data_ptr(), buf.data_ptr() + 3072, 1, 0) \
        == hefx.HEFX_EUNSUPPORTED
    hefx.hefx_params_set_reduction(ctx, p3, "shoup", "montgomery")
    assert hefx.raw_status("hefx_key_inner_product", ctx, p3, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 0, 1,
                           0) == hefx.HEFX_EINVAL
    plan = hefx.hefx_bconv_plan_create(ctx, 8, inputs.special_primes(1), inputs.source_primes(2))
    # ModDown output overlapping its input
    assert hefx.raw_status("hefx_mod_down", ctx, plan, buf.data_ptr(), buf.data_ptr() + 1024, 1, 0) \
        == hefx.HEFX_EINVAL
    hefx.hefx_bconv_plan_destroy(plan)
    hefx.hefx_params_destroy(p1)
    hefx.hefx_params_destroy(p3)


def _he_mult_case(logn, L, K, alpha, seed, genuine_key):
    n = 1 << logn
    qs, ps = inputs.source_primes(L), inputs.special_primes(K)
    qp = list(qs) + list(ps)
    dn = len(oks.digit_ranges(L, alpha))
    s = None
    if genuine_key:
        s = np.random.default_rng(seed).integers(-1, 2, n)
        a_r = np.stack([_res((seed, 1, j), 1, qp, n)[0] for j in range(dn)])
        evk = oks.keygen(s, qs, ps, alpha, a_r)
    else:
        evk = np.stack([np.stack([_res((seed, 3, j, k), 1, qp, n)[0] for k in range(2)]) for j in range(dn)])
    ins = [_res((seed, 2, c), 1, qs, n)[0] for c in range(4)]
    return qs, ps, s, evk, ins


@pytest.mark.parametrize("logn,L,K,alpha,genuine,bconv", [(6, 5, 2, 2, True, "auto"), (10, 6, 3, 3, True, "auto"),
                                                           (8, 4, 4, 4, True, "auto"), (16, 24, 8, 8, False, "auto"),
                                                           (16, 48, 16, 16, False, "auto"),
                                                           (10, 6, 3, 3, True, "tensor")])
def test_he_mult_matches_oracle(hx, logn, L, K, alpha, genuine, bconv):
    """bconv "auto": one-launch ModUp; "tensor": per-digit conversions on the tensor path.
    (16, 48, 16, 16) is the shape bench.py times: (L, log q, dnum) = (48, 28, 3), K = 16."""
    hefx, ctx = hx
    from paper_2501_07047_gb300.hemult import HeMult
    qs, ps, s, evk, ins = _he_mult_case(logn, L, K, alpha, 64 + logn, genuine)
    hm = HeMult(ctx, logn, qs, ps, alpha, bconv_path=bconv)
    n = 1 << logn
    out = dev(np.zeros((2, L - 1, n), dtype=np.uint32))
    dins = [dev(a) for a in ins]
    devk = dev(evk)
    hm.run(*dins, devk, out)
    want = oks.he_mult(*ins, evk, qs, ps, alpha)
    got = host(out)
    assert np.array_equal(got[0], want["c0r"]) and np.array_equal(got[1], want["c1r"])
    st = {k: host(v) for k, v in hm.stages().items()}
    qp = list(qs) + list(ps)
    assert np.array_equal(st["d2_coeff"], oracle.ntt_batch(want["d2"][None], qs, inverse=True)[0])
    assert np.array_equal(st["modup_eval"], oracle.ntt_batch(want["modup"], qp))
    assert np.array_equal(st["acc_coeff"], oracle.ntt_batch(want["acc"], qp, inverse=True))
    assert np.array_equal(st["ks_eval"], oracle.ntt_batch(want["ks"], qs))
    if genuine:
        res = dict(want, c0r=got[0], c1r=got[1])
        assert oks.phase_error(res, s, qs) <= 2 * n + 2 * K + 8
    hm.close()


def test_he_mult_graph_replay(hx):
    """The HE-Mult sequence captured as one CUDA graph replays to the oracle's result."""
    import torch
    hefx_, ctx = hx
    from paper_2501_07047_gb300.hemult import HeMult
    logn, L, K, alpha = 12, 6, 3, 3
    qs, ps, s, evk, ins = _he_mult_case(logn, L, K, alpha, 90, True)
    hm = HeMult(ctx, logn, qs, ps, alpha)
    out = dev(np.zeros((2, L - 1, 1 << logn), dtype=np.uint32))
    dins = [dev(a) for a in ins]
    devk = dev(evk)
    g = hm.capture(*dins, devk, out)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    want = oks.he_mult(*ins, evk, qs, ps, alpha)
    got = host(out)
    assert np.array_equal(got[0], want["c0r"]) and np.array_equal(got[1], want["c1r"])
    del g
    hm.close()
