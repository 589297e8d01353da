"""Host-side logic that needs no GPU: key-switching digit ranges, the bench's traffic-file
reader and its source-hash check, the path tuner's cache, and the seeded input generators."""
import hashlib
import importlib.util
import json
import os

import numpy as np
import pytest

from oracle import keyswitch as oks
from paper_2501_07047_gb300 import inputs
from paper_2501_07047_gb300.hemult import digit_ranges

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("L,alpha", [(1, 1), (5, 2), (6, 3), (7, 7), (48, 16), (24, 8), (10, 4)])
def test_digit_ranges_partition(L, alpha):
    """HE-Mult's digits equal the oracle's and partition [0, L) into ceil(L / alpha) ranges."""
    d = digit_ranges(L, alpha)
    assert d == oks.digit_ranges(L, alpha)
    assert len(d) == -(-L // alpha)
    assert d[0][0] == 0 and d[-1][1] == L
    assert all(a < b <= a + alpha for a, b in d)
    assert all(d[i][1] == d[i + 1][0] for i in range(len(d) - 1))


def test_profile_traffic_reader(tmp_path):
    """The committed traffic figures are read only while the kernel source still matches."""
    b = _bench()
    fwd, inv = b.profile_traffic("ntt_cc", "fwd"), b.profile_traffic("ntt_cc", "inv")
    assert fwd is not None and inv is not None and 48 << 20 < fwd < 80 << 20 and 48 << 20 < inv < 80 << 20
    # a copy of the tree whose kernel source differs: no traffic figure
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_2501_07047_gb300" / "csrc").mkdir(parents=True)
    text = open(os.path.join(ROOT, "profiles", "ntt_cc_traffic.txt")).read()
    (tmp_path / "profiles" / "ntt_cc_traffic.txt").write_text(text)
    src = tmp_path / "paper_2501_07047_gb300" / "csrc" / "ntt_cc_impl.cuh"
    src.write_text("// changed\n")
    b.ROOT = str(tmp_path)
    assert b.profile_traffic("ntt_cc", "fwd") is None
    # and with a matching hash the figure comes back
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    lines = [("source_sha=" + sha) if ln.startswith("source_sha=") else ln for ln in text.split("\n")]
    (tmp_path / "profiles" / "ntt_cc_traffic.txt").write_text("\n".join(lines))
    assert b.profile_traffic("ntt_cc", "fwd") == fwd
    assert b.profile_traffic("ntt_cc", "nope") is None


def test_tuner_cache_round_trip(tmp_path, monkeypatch):
    from paper_2501_07047_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "sub" / "tune.json"))
    assert autotune._load_cache() == {}
    autotune._save_cache({"GB300|16|24": "cudacore"})
    assert autotune._load_cache() == {"GB300|16|24": "cudacore"}
    assert json.load(open(tmp_path / "sub" / "tune.json")) == {"GB300|16|24": "cudacore"}


def test_input_generators():
    """Seeded and reproducible; residues below their prime; primes prime and NTT-friendly."""
    assert inputs.derive_seed(2, 0) == inputs.derive_seed(2, 0) != inputs.derive_seed(2, 1)
    qs = inputs.source_primes(6)
    a = inputs.residue_tensor(inputs.derive_seed(7, 1), 2, qs, 1 << 10)
    assert a.shape == (2, 6, 1 << 10) and a.dtype == np.uint32
    assert np.array_equal(a, inputs.residue_tensor(inputs.derive_seed(7, 1), 2, qs, 1 << 10))
    assert (a < np.asarray(qs, dtype=np.uint32)[None, :, None]).all()
    for q in qs + inputs.special_primes(4) + inputs.ntt_primes(3, 28, 1 << 18):
        assert q % 2 and all(q % d for d in range(3, int(q ** 0.5) + 1, 2))  # trial division (q < 2^30)
    assert all(q % (1 << 17) == 1 and q < (1 << 28) for q in qs)
    assert all(p % (1 << 17) == 1 and (1 << 29) < p < (1 << 30) for p in inputs.special_primes(4))
    assert all(q % (1 << 18) == 1 for q in inputs.ntt_primes(3, 28, 1 << 18))
    t = inputs.poisson_arrivals(inputs.derive_seed(5, 1), 500, 1000.0)
    assert np.all(np.diff(t) >= 0) and 0.2 < t[-1] < 1.0  # about 0.5 s of arrivals at 1000/s


def test_tensor_work_model():
    """The tensor path's roofline numerator: 2 flops per digit MAC, 4 x 4 digit products per
    modular product, N (R + C) modular MACs per limb-NTT for the square split (1.074 GFLOP at
    N = 2^16), and the 7-bit digits' worst-case partial sum stays exact in fp32."""
    from paper_2501_07047_gb300 import tensor_plan as tp
    assert tp.split(16) == (256, 256) and tp.split(15) == (128, 256) and tp.split(14) == (128, 128)
    assert tp.flops_per_limb_ntt(16) == 2 * 4 * 4 * 65536 * 512 == 1073741824
    assert tp.flops_per_step_launch(16, 192) * 2 == tp.flops_per_limb_ntt(16) * 192
    R, _ = tp.split(16)
    worst = tp.K_IN * R * ((1 << tp.W_IN) - 1) * ((1 << tp.W_OUT) - 1)  # one output's digit sum
    assert worst < (1 << 24)  # every partial sum is an exact fp32 integer
    assert tp.K_IN * tp.W_IN >= 28  # four 7-bit digits hold a 28-bit residue


def test_tuner_candidates_and_cached_choice(tmp_path, monkeypatch):
    """The tuner's search space (path x split x tile) and its cache: a measured winner is
    stored per shape and batch and reapplied without timing again."""
    import torch
    from paper_2501_07047_gb300 import autotune, tensor_plan
    assert [s for s in tensor_plan.splits(15) if not s[1]] == [(7, 0), (8, 0)]
    assert [s for s in tensor_plan.splits(16) if not s[1]] == [(8, 0)]
    assert tensor_plan.tuned_splits(16) == [(8, 0), (6, 5)]            # 256 x 256 and 64 x 32 x 32
    assert tensor_plan.tuned_splits(14) == [(6, 0), (7, 0), (8, 0), (6, 4)]  # 64 x 256 .. 256 x 64, 64 x 16 x 16
    assert tensor_plan.splits(13) == [(6, 0), (7, 0)] and tensor_plan.splits(12) == [(6, 0)]
    assert tensor_plan.splits(11) == []
    # 8-bit digits (moduli of 29-30 bits): exact fp32 sums need every factor <= 64
    assert tensor_plan.splits_wide(16) == [(6, 4), (6, 5), (6, 6)]
    assert tensor_plan.splits_wide(15) == [(6, 4), (6, 5)] and tensor_plan.splits_wide(14) == [(6, 4)]
    assert tensor_plan.splits_wide(13) == [] and tensor_plan.splits_wide(12) == [(6, 0)]
    assert 4 * tensor_plan.MAX_FACTOR_WIDE * 255 * 255 < 2 ** 24 < 4 * 2 * tensor_plan.MAX_FACTOR_WIDE * 255 * 255
    assert autotune.candidates(11) == [("cudacore", 0, 0, 0)]
    assert autotune.candidates(16)[:2] == [("cudacore", 1, 0, 0), ("cudacore", 2, 0, 0)]  # both schedules
    assert autotune.candidates(15)[0] == ("cudacore", 0, 0, 0) and autotune.candidates(15)[1][0] == "tensor"
    for logn in (12, 13, 14, 15, 16):
        for log2r, log2r2 in tensor_plan.splits(logn):  # every split multiplies out to N within bounds
            f = tensor_plan.split(logn, log2r, log2r2)
            assert int(np.prod(f)) == 1 << logn
            if log2r2:
                assert 64 <= f[0] <= 256 and all(16 <= x <= 256 for x in f[1:])
            else:
                assert all(x in (64, 128, 256) for x in f)
        for cand in autotune.candidates(logn)[2 if logn == 16 else 1:]:
            assert cand[0] == "tensor" and cand[3] in autotune.TILES
            assert autotune.parse(autotune.key_of(cand)) == cand
    # digit MACs: the three-factor split costs (R1 + R2 + R3) / (R + C) of the two-factor one
    assert tensor_plan.flops_per_limb_ntt(16, 6, 5) * 4 == tensor_plan.flops_per_limb_ntt(16)
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FAKE-GPU")
    timed, applied = [], []
    monkeypatch.setattr(autotune, "time_candidates",
                        lambda *a, **k: timed.append(1) or {"cudacore/1/0/0": 2.0, "cudacore/2/0/0": 2.1, "tensor/6/5/32": 1.5,
                                                            "tensor/8/0/64": 1.7})
    monkeypatch.setattr(autotune, "apply", lambda ctx, p, cand: applied.append(cand))
    assert autotune.tune(None, None, 16, [268042241, 265420801]) == "tensor"
    assert applied[-1] == ("tensor", 6, 5, 32) and len(timed) == 1
    assert autotune.tune(None, None, 16, [268042241, 265420801]) == "tensor"  # from the cache
    assert applied[-1] == ("tensor", 6, 5, 32) and len(timed) == 1
    assert autotune.tune(None, None, 16, [268042241, 265420801], batch=8) == "tensor"  # another batch: timed
    assert len(timed) == 2
