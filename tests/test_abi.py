"""The C-ABI library builds, loads and exports every symbol include/hefx.h declares (no GPU)."""
import os
import re

import pytest

from paper_2501_07047_gb300 import build, hefx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hefx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hefx_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("hefx_ntt_fwd", "hefx_ntt_inv", "hefx_poly_mul", "hefx_basis_convert", "hefx_create",
                 "hefx_params_create", "hefx_bconv_plan_create"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    lib = hefx.load(build.build())
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) == set(hefx.SIGNATURES)


def test_version_string():
    assert "sm_103a" in hefx.hefx_version()


def test_no_gpu_create_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hefx.HefxError):
        hefx.hefx_create(0)
