"""GPU parity of the NTT / INTT / polynomial product against the CPU oracle, through the C ABI.

Integer work: every comparison is bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_2501_07047_gb300 import hefx, inputs

from hefx_testutil import empty_dev, to_dev, to_host

pytestmark = pytest.mark.gpu

PATHS = ["cudacore", "tensor"]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = hefx.hefx_create(0)
    yield c
    hefx.hefx_destroy(c)


def make_params(ctx, logn, primes):
    return hefx.hefx_params_create(ctx, logn, primes)


def run_fwd(ctx, params, arr, path):
    d = to_dev(arr)
    hefx.hefx_ntt_fwd(ctx, params, d, arr.shape[0], path)
    hefx.hefx_stream_check(ctx, params)
    return to_host(d).reshape(arr.shape)


def run_inv(ctx, params, arr, path):
    d = to_dev(arr)
    hefx.hefx_ntt_inv(ctx, params, d, arr.shape[0], path)
    hefx.hefx_stream_check(ctx, params)
    return to_host(d).reshape(arr.shape)


def supported(ctx, params, path, batch=1, L=1, n=8):
    if path == "cudacore":
        return True
    d = empty_dev((batch, L, n))
    st = hefx.raw_status("hefx_ntt_fwd", ctx, params, d.data_ptr(), 0, hefx.PATHS[path], 0)
    return st == hefx.HEFX_OK


# ----------------------------------------------------------------------------- config 1

def test_config1_single_limb_cudacore(ctx):
    """N = 4096, one 28-bit prime q = 1 mod 8192: forward, inverse and one product."""
    q = inputs.source_primes(1)[0]
    assert (q - 1) % 8192 == 0
    p = make_params(ctx, 12, [q])
    try:
        a = inputs.uniform_residues(inputs.derive_seed(1, 1), 4096, q)
        b = inputs.uniform_residues(inputs.derive_seed(1, 2), 4096, q)
        ahat = run_fwd(ctx, p, a.reshape(1, 1, -1), "cudacore")[0, 0]
        assert (ahat == oracle.ntt(a, q)).all()
        back = run_inv(ctx, p, ahat.reshape(1, 1, -1), "cudacore")[0, 0]
        assert (back == a).all()
        da, db, dc = to_dev(a), to_dev(b), empty_dev(4096)
        hefx.hefx_poly_mul(ctx, p, da, db, dc, 1, "cudacore")
        c = to_host(dc)
        assert (c == oracle.polymul_schoolbook(a, b, q)).all()
    finally:
        hefx.hefx_params_destroy(p)


# ----------------------------------------------------------------------------- shapes

@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("logn,L,batch", [(3, 1, 1), (4, 3, 5), (5, 2, 3), (6, 1, 7), (7, 5, 2), (8, 3, 3),
                                          (9, 2, 2), (10, 4, 3), (11, 3, 1), (12, 5, 3), (13, 2, 3),
                                          (14, 3, 2), (15, 2, 2), (16, 3, 2)])
def test_ntt_matches_oracle(ctx, path, logn, L, batch):
    primes = inputs.source_primes(L + 2)[2:]
    p = make_params(ctx, logn, primes)
    try:
        if not supported(ctx, p, path, batch, L, 1 << logn):
            pytest.skip(f"{path} path not built for N = 2^{logn}")
        data = inputs.residue_tensor(inputs.derive_seed(10, logn, L, batch), batch, primes, 1 << logn)
        expect = oracle.ntt_batch(data, primes)
        got = run_fwd(ctx, p, data, path)
        assert (got == expect).all(), f"first mismatch at {np.argwhere(got != expect)[0]}"
        back = run_inv(ctx, p, got, path)
        assert (back == data).all()
        # the inverse alone against the oracle on an arbitrary (not forward-produced) input
        rnd = inputs.residue_tensor(inputs.derive_seed(11, logn, L, batch), batch, primes, 1 << logn)
        assert (run_inv(ctx, p, rnd, path) == oracle.ntt_batch(rnd, primes, inverse=True)).all()
    finally:
        hefx.hefx_params_destroy(p)


@pytest.mark.parametrize("path", PATHS)
def test_special_primes_30bit(ctx, path):
    primes = inputs.special_primes(3)
    p = make_params(ctx, 16, primes)
    try:
        if not supported(ctx, p, path, 1, 3, 1 << 16):
            pytest.skip("path not built for 30-bit moduli")
        data = inputs.residue_tensor(21, 1, primes, 1 << 16)
        got = run_fwd(ctx, p, data, path)
        assert (got == oracle.ntt_batch(data, primes)).all()
        assert (run_inv(ctx, p, got, path) == data).all()
    finally:
        hefx.hefx_params_destroy(p)


@pytest.mark.parametrize("path", PATHS)
def test_edge_values(ctx, path):
    """All-zero, all q-1 (the largest residue) and a delta input."""
    primes = inputs.source_primes(2)
    n = 1 << 16
    p = make_params(ctx, 16, primes)
    try:
        if not supported(ctx, p, path, 3, 2, n):
            pytest.skip("path not built")
        data = np.zeros((3, 2, n), np.uint32)
        for l, q in enumerate(primes):
            data[1, l, :] = q - 1
            data[2, l, 0] = 1
        got = run_fwd(ctx, p, data, path)
        assert (got[0] == 0).all()
        assert (got[2] == 1).all()
        assert (got == oracle.ntt_batch(data, primes)).all()
        assert (run_inv(ctx, p, got, path) == data).all()
    finally:
        hefx.hefx_params_destroy(p)


# ----------------------------------------------------------------------------- config 2 (full size)

def oracle_rows(data, primes, inverse=False):
    """oracle.ntt_batch over the polynomials of `data`, one thread per polynomial (the oracle's
    C calls release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=8) as ex:
        parts = list(ex.map(lambda b: oracle.ntt_batch(data[b:b + 1], primes, inverse=inverse), range(len(data))))
    return np.concatenate(parts)


@pytest.mark.parametrize("path,schedule", [("cudacore", "cluster"), ("cudacore", "two_pass"), ("tensor", "auto")])
def test_config2_full_size(ctx, path, schedule):
    """N = 2^16, L = 24, batch 8 (192 limb-NTTs, the bench launch), on both CUDA-core schedules
    and the tensor path: every output of the forward transform and of the inverse of an
    arbitrary input against the oracle, 256 sampled forward outputs against the O(N) definition
    (pinning the oracle itself at full size), and INTT(NTT(x)) = x over the whole batch."""
    primes = inputs.source_primes(24)
    n = 1 << 16
    p = make_params(ctx, 16, primes)
    try:
        if not supported(ctx, p, path, 8, 24, n):
            pytest.skip("path not built")
        hefx.hefx_params_set_cc_schedule(ctx, p, schedule)
        data = inputs.residue_tensor(inputs.derive_seed(2, 0), 8, primes, n)
        d = to_dev(data)
        hefx.hefx_ntt_fwd(ctx, p, d, 8, path)
        hefx.hefx_stream_check(ctx, p)
        got = to_host(d).reshape(data.shape)
        want = oracle_rows(data, primes)
        bad = np.argwhere(got != want)
        assert bad.size == 0, f"{len(bad)} forward outputs differ, first at {bad[0]}"
        rng = np.random.default_rng(5)
        for _ in range(256):
            b, l, k = int(rng.integers(8)), int(rng.integers(24)), int(rng.integers(n))
            assert want[b, l, k] == oracle.ntt_at(data[b, l], primes[l], k)
        hefx.hefx_ntt_inv(ctx, p, d, 8, path)
        assert (to_host(d).reshape(data.shape) == data).all()
        rnd = inputs.residue_tensor(inputs.derive_seed(2, 1), 8, primes, n)
        d = to_dev(rnd)
        hefx.hefx_ntt_inv(ctx, p, d, 8, path)
        hefx.hefx_stream_check(ctx, p)
        got = to_host(d).reshape(rnd.shape)
        bad = np.argwhere(got != oracle_rows(rnd, primes, inverse=True))
        assert bad.size == 0, f"{len(bad)} inverse outputs differ, first at {bad[0]}"
    finally:
        hefx.hefx_params_destroy(p)


@pytest.mark.parametrize("bits,L,batch", [(28, 1, 1), (28, 5, 3), (30, 3, 1), (30, 2, 20), (28, 24, 5)])
def test_cc_schedules_agree_with_oracle(ctx, bits, L, batch):
    """The two CUDA-core schedules at N = 2^16 (cluster, two-pass) and AUTO (two-pass up to 32
    rows and between one and one and a half waves of clusters, cluster elsewhere): every output
    of the forward and inverse transforms against the oracle, for 28-bit moduli (lazy ranges)
    and 30-bit ones (Harvey ranges), from one row to 120 rows (inside the second AUTO band on
    GB300's 89 co-resident clusters)."""
    primes = inputs.source_primes(L) if bits == 28 else inputs.special_primes(L)
    n = 1 << 16
    p = make_params(ctx, 16, primes)
    try:
        data = inputs.residue_tensor(inputs.derive_seed(15, bits, L, batch), batch, primes, n)
        want_f = oracle_rows(data, primes)
        want_i = oracle_rows(data, primes, inverse=True)
        for schedule in ("cluster", "two_pass", "auto"):
            hefx.hefx_params_set_cc_schedule(ctx, p, schedule)
            got = run_fwd(ctx, p, data, "cudacore")
            bad = np.argwhere(got != want_f)
            assert bad.size == 0, f"{schedule}: {len(bad)} forward outputs differ, first at {bad[0]}"
            got = run_inv(ctx, p, data, "cudacore")
            bad = np.argwhere(got != want_i)
            assert bad.size == 0, f"{schedule}: {len(bad)} inverse outputs differ, first at {bad[0]}"
    finally:
        hefx.hefx_params_destroy(p)


def test_cc_schedule_validation(ctx):
    p = make_params(ctx, 15, inputs.source_primes(2))
    try:
        with pytest.raises(hefx.HefxError) as e:
            hefx.hefx_params_set_cc_schedule(ctx, p, "two_pass")  # built for N = 2^16 only
        assert e.value.status == hefx.HEFX_EUNSUPPORTED
        hefx.hefx_params_set_cc_schedule(ctx, p, "cluster")
        hefx.hefx_params_set_cc_schedule(ctx, p, "auto")
        assert hefx.raw_status("hefx_params_set_cc_schedule", p, 7) == hefx.HEFX_EINVAL
    finally:
        hefx.hefx_params_destroy(p)


# ----------------------------------------------------------------------------- products

@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("logn,L,batch", [(3, 2, 2), (6, 1, 3), (10, 3, 2), (12, 2, 2), (13, 2, 1), (15, 2, 1),
                                          (16, 3, 2)])
def test_poly_mul_matches_oracle(ctx, path, logn, L, batch):
    primes = inputs.source_primes(L)
    n = 1 << logn
    p = make_params(ctx, logn, primes)
    try:
        if not supported(ctx, p, path, batch, L, n):
            pytest.skip("path not built")
        a = inputs.residue_tensor(inputs.derive_seed(30, logn), batch, primes, n)
        b = inputs.residue_tensor(inputs.derive_seed(31, logn), batch, primes, n)
        expect = oracle.polymul_batch(a, b, primes)
        if logn <= 10:
            for l, q in enumerate(primes):
                assert (expect[0, l] == oracle.polymul_schoolbook(a[0, l], b[0, l], q)).all()
        da, db, dc = to_dev(a), to_dev(b), empty_dev(a.shape)
        hefx.hefx_poly_mul(ctx, p, da, db, dc, batch, path)
        hefx.hefx_stream_check(ctx, p)
        assert (to_host(dc).reshape(a.shape) == expect).all()
        # aliasing: c = a, c = b, a = b (square), a = b = c
        hefx.hefx_poly_mul(ctx, p, da, db, da, batch, path)
        assert (to_host(da).reshape(a.shape) == expect).all()
        da = to_dev(a)
        hefx.hefx_poly_mul(ctx, p, da, db, db, batch, path)
        assert (to_host(db).reshape(a.shape) == expect).all()
        sq = oracle.polymul_batch(a, a, primes)
        da, dc = to_dev(a), empty_dev(a.shape)
        hefx.hefx_poly_mul(ctx, p, da, da, dc, batch, path)
        assert (to_host(dc).reshape(a.shape) == sq).all()
        hefx.hefx_poly_mul(ctx, p, da, da, da, batch, path)
        assert (to_host(da).reshape(a.shape) == sq).all()
    finally:
        hefx.hefx_params_destroy(p)


# ----------------------------------------------------------------------------- errors

def test_host_validation(ctx):
    q = inputs.source_primes(1)[0]
    with pytest.raises(hefx.HefxError) as e:
        hefx.hefx_params_create(ctx, 12, [q + 2])          # not prime
    assert e.value.status == hefx.HEFX_EINVAL
    with pytest.raises(hefx.HefxError) as e:
        hefx.hefx_params_create(ctx, 12, [7681])           # prime but not 1 mod 2N for N = 4096
    assert e.value.status == hefx.HEFX_EINVAL
    with pytest.raises(hefx.HefxError) as e:
        hefx.hefx_params_create(ctx, 12, [q, q])           # repeated
    assert e.value.status == hefx.HEFX_EINVAL
    with pytest.raises(hefx.HefxError) as e:
        hefx.hefx_params_create(ctx, 18, [q])
    assert e.value.status == hefx.HEFX_EUNSUPPORTED
    p = hefx.hefx_params_create(ctx, 12, [q])
    try:
        d = empty_dev(4096 + 4)
        with pytest.raises(hefx.HefxError) as e:
            hefx.hefx_ntt_fwd(ctx, p, d.data_ptr() + 4, 1)  # misaligned
        assert e.value.status == hefx.HEFX_EINVAL
        with pytest.raises(hefx.HefxError):
            hefx.hefx_ntt_fwd(ctx, p, 0, 1)
        hefx.hefx_ntt_fwd(ctx, p, d, 0)                     # batch 0: no-op
    finally:
        hefx.hefx_params_destroy(p)


@pytest.mark.parametrize("logn", [15, 16])
def test_autotune_sets_auto_path(ctx, tmp_path, monkeypatch, logn):
    """The tuner measures every candidate (path, split, tile), caches the winner and applies
    it; AUTO then runs it bit-exactly."""
    import json
    from paper_2501_07047_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    primes = inputs.source_primes(4)
    p = make_params(ctx, logn, primes)
    try:
        best = autotune.tune(ctx, p, logn, primes)
        assert best in ("cudacore", "tensor")
        entry = next(iter(json.load(open(tmp_path / "tune.json")).values()))
        assert set(entry["ms"]) == {autotune.key_of(c) for c in autotune.candidates(logn)}
        data = inputs.residue_tensor(inputs.derive_seed(12, logn), 2, primes, 1 << logn)
        assert (run_fwd(ctx, p, data, "auto") == oracle.ntt_batch(data, primes)).all()
    finally:
        hefx.hefx_params_destroy(p)


@pytest.mark.parametrize("logn", [12, 13, 14, 15, 16])
def test_tensor_configs_bit_exact(ctx, logn):
    """Every tensor-path split (two factors, and every three-factor split) with both tile widths
    gives the oracle's transforms and products; invalid splits and tiles are refused."""
    from paper_2501_07047_gb300 import tensor_plan
    primes = inputs.source_primes(3)
    n = 1 << logn
    p = make_params(ctx, logn, primes)
    try:
        a = inputs.residue_tensor(inputs.derive_seed(13, logn, 0), 2, primes, n)
        b = inputs.residue_tensor(inputs.derive_seed(13, logn, 1), 2, primes, n)
        want_f = oracle.ntt_batch(a, primes)
        want_m = oracle.polymul_batch(a, b, primes)
        for log2r, log2r2 in tensor_plan.splits(logn):
            for tile in (64, 32):
                hefx.hefx_params_set_tensor_config(ctx, p, log2r, tile, log2r2)
                got = run_fwd(ctx, p, a, "tensor")
                assert (got == want_f).all(), (log2r, log2r2, tile)
                assert (run_inv(ctx, p, got, "tensor") == a).all(), (log2r, log2r2, tile)
                rnd = inputs.residue_tensor(inputs.derive_seed(14, logn), 1, primes, n)
                assert (run_inv(ctx, p, rnd, "tensor") == oracle.ntt_batch(rnd, primes, inverse=True)).all()
                da, db, dc = to_dev(a), to_dev(b), empty_dev(a.shape)
                hefx.hefx_poly_mul(ctx, p, da, db, dc, 2, "tensor")
                hefx.hefx_stream_check(ctx, p)
                assert (to_host(dc).reshape(a.shape) == want_m).all(), (log2r, log2r2, tile)
        for bad in ((logn // 2 - 2, 64, 0), (0, 48, 0), (5, 64, 5), (6, 64, 3)):
            with pytest.raises(hefx.HefxError) as e:
                hefx.hefx_params_set_tensor_config(ctx, p, bad[0], bad[1], bad[2])
            assert e.value.status == hefx.HEFX_EINVAL
    finally:
        hefx.hefx_params_destroy(p)

# ----------------------------------------------------------------------------- N = 2^17

@pytest.mark.parametrize("logn", [12, 14, 15, 16])
def test_tensor_30bit_moduli(ctx, logn):
    """Moduli of 29-30 bits on the tensor path (8-bit digits and chunks): every split it
    accepts (every factor at most 64: 64 x 64 at 2^12, three factors above) with both tile
    widths gives the oracle's forward and inverse transforms and products; splits with a
    larger factor are refused, as is the single-pass no-allocation product; N = 2^13 (no such
    split) stays on the CUDA cores."""
    from paper_2501_07047_gb300 import tensor_plan
    primes = inputs.special_primes(3)
    n = 1 << logn
    p = make_params(ctx, logn, primes)
    try:
        a = inputs.residue_tensor(inputs.derive_seed(16, logn, 0), 2, primes, n)
        b = inputs.residue_tensor(inputs.derive_seed(16, logn, 1), 2, primes, n)
        # extreme residues: q - 1 everywhere in one limb
        a[1, 2, :] = primes[2] - 1
        want_f = oracle.ntt_batch(a, primes)
        want_m = oracle.polymul_batch(a, b, primes)
        rnd = inputs.residue_tensor(inputs.derive_seed(17, logn), 1, primes, n)
        want_i = oracle.ntt_batch(rnd, primes, inverse=True)
        # the default split of a 30-bit parameter set
        assert (run_fwd(ctx, p, a, "tensor") == want_f).all()
        for log2r, log2r2 in tensor_plan.splits_wide(logn):
            for tile in (64, 32):
                hefx.hefx_params_set_tensor_config(ctx, p, log2r, tile, log2r2)
                got = run_fwd(ctx, p, a, "tensor")
                assert (got == want_f).all(), (log2r, log2r2, tile)
                assert (run_inv(ctx, p, got, "tensor") == a).all(), (log2r, log2r2, tile)
                assert (run_inv(ctx, p, rnd, "tensor") == want_i).all(), (log2r, log2r2, tile)
                da, db, dc = to_dev(a), to_dev(b), empty_dev(a.shape)
                hefx.hefx_poly_mul(ctx, p, da, db, dc, 2, "tensor")
                assert (to_host(dc).reshape(a.shape) == want_m).all(), (log2r, log2r2, tile)
        if logn >= 14:
            with pytest.raises(hefx.HefxError) as e:
                hefx.hefx_params_set_tensor_config(ctx, p, logn // 2, 64, 0)
            assert e.value.status == hefx.HEFX_EUNSUPPORTED
        if logn >= 15:
            with pytest.raises(hefx.HefxError) as e:  # a factor above 64
                hefx.hefx_params_set_tensor_config(ctx, p, 7, 64, 4)
            assert e.value.status == hefx.HEFX_EUNSUPPORTED
        d = to_dev(a)
        assert hefx.raw_status("hefx_poly_mul_noalloc", ctx, p, d.data_ptr(), d.data_ptr(), d.data_ptr(), 2, None) \
            == hefx.HEFX_EUNSUPPORTED
    finally:
        hefx.hefx_params_destroy(p)
    p13 = make_params(ctx, 13, primes)
    try:
        assert not supported(ctx, p13, "tensor", 1, 3, 1 << 13)
    finally:
        hefx.hefx_params_destroy(p13)


@pytest.mark.parametrize("bits", [28, 30])
def test_n_2_17(ctx, bits):
    """N = 2^17 (primes = 1 mod 2^18) on the CUDA cores: 28-bit moduli take the lazy
    butterflies, 30-bit ones Harvey's; forward, inverse and product against the oracle."""
    logn, L, batch = 17, 3, 2
    n = 1 << logn
    primes = inputs.ntt_primes(L, bits, two_n=1 << 18)
    p = make_params(ctx, logn, primes)
    try:
        a = inputs.residue_tensor(inputs.derive_seed(32, bits, 0), batch, primes, n)
        b = inputs.residue_tensor(inputs.derive_seed(32, bits, 1), batch, primes, n)
        got = run_fwd(ctx, p, a, "cudacore")
        assert (got == oracle.ntt_batch(a, primes)).all()
        assert (run_inv(ctx, p, got, "cudacore") == a).all()
        da, db, dc = to_dev(a), to_dev(b), empty_dev(a.shape)
        hefx.hefx_poly_mul(ctx, p, da, db, dc, batch, "cudacore")
        hefx.hefx_stream_check(ctx, p)
        assert (to_host(dc).reshape(a.shape) == oracle.polymul_batch(a, b, primes)).all()
        # the tensor path is not built for N = 2^17: it refuses instead of computing
        d = empty_dev((1, L, n))
        assert hefx.raw_status("hefx_ntt_fwd", ctx, p, d.data_ptr(), 1, hefx.PATHS["tensor"], 0) \
            == hefx.HEFX_EUNSUPPORTED
    finally:
        hefx.hefx_params_destroy(p)


def test_large_batch_sampled(ctx):
    """A large launch (2048 rows of N = 2^16, 512 MiB: 16k CTAs in 2048 clusters) on the
    CUDA-core path: sampled rows against the oracle, every row through the round trip."""
    import torch
    logn, L, batch = 16, 32, 64
    n = 1 << logn
    primes = inputs.source_primes(L)
    p = make_params(ctx, logn, primes)
    try:
        small = inputs.residue_tensor(inputs.derive_seed(33, 0), 2, primes, n)
        d = torch.from_numpy(np.tile(small, (batch // 2, 1, 1)).view(np.int32)).cuda()
        d0 = d.clone()
        hefx.hefx_ntt_fwd(ctx, p, d, batch, "cudacore")
        hefx.hefx_stream_check(ctx, p)
        got = to_host(d).reshape(batch, L, n)
        want = oracle.ntt_batch(small, primes)
        for b in (0, 1, batch // 2, batch - 1):  # identical inputs in every pair of polynomials
            assert (got[b] == want[b % 2]).all()
        hefx.hefx_ntt_inv(ctx, p, d, batch, "cudacore")
        hefx.hefx_stream_check(ctx, p)
        assert torch.equal(d, d0)
    finally:
        hefx.hefx_params_destroy(p)


@pytest.mark.parametrize("path", PATHS)
def test_overlapping_streams(ctx, path):
    """Independent batches whose transforms overlap on two streams (the benchmark's whole-job
    loop): the CUDA-core path shares one parameter set between the streams, the tensor path
    takes one per stream (its digit workspace lives in the parameter set).  Every forward
    result equals the oracle's and every round trip returns its batch."""
    import torch
    L, B, logn = 24, 3, 16
    n = 1 << logn
    primes = inputs.source_primes(L)
    nparams = 2 if path == "tensor" else 1
    params = [make_params(ctx, logn, primes) for _ in range(nparams)]
    try:
        if hefx.raw_status("hefx_ntt_fwd", ctx, params[0], empty_dev((1, L, n)).data_ptr(), 0,
                           hefx.PATHS[path], 0) != hefx.HEFX_OK:
            pytest.skip(f"{path} path not built at N = 2^{logn}")
        host = [inputs.residue_tensor(inputs.derive_seed(43, k), B, primes, n) for k in range(4)]
        bufs = [to_dev(h) for h in host]
        fwd = [empty_dev((B, L, n)) for _ in range(4)]
        streams = [torch.cuda.Stream() for _ in range(2)]
        torch.cuda.synchronize()
        for rep in range(3):
            for k in range(4):
                s, p = streams[k % 2], params[k % nparams]
                hefx.hefx_ntt_fwd(ctx, p, bufs[k], B, path, s)
                if rep == 0:
                    with torch.cuda.stream(s):
                        fwd[k].copy_(bufs[k])
                hefx.hefx_ntt_inv(ctx, p, bufs[k], B, path, s)
        torch.cuda.synchronize()
        for p in params:
            hefx.hefx_stream_check(ctx, p)
        for k in range(4):
            assert (to_host(bufs[k]).reshape(host[k].shape) == host[k]).all(), k
        for k in (0, 3):
            assert (to_host(fwd[k]).reshape(host[k].shape) == oracle.ntt_batch(host[k], primes)).all(), k
    finally:
        for p in params:
            hefx.hefx_params_destroy(p)
