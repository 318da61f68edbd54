"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/dpd.h declares; the Python binding wraps exactly those names.  No compute
call is made (these run on machines without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1807_09896_gb300 import _build, dpd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dpd.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dpd_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    return _build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["dpd_create", "dpd_set_phase_field", "dpd_set_particles", "dpd_step",
                 "dpd_get_state", "dpd_velocity_profile", "dpd_destroy", "dpd_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (dpd_[a-z_]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    L = ctypes.CDLL(lib_path)
    for n in _declared():
        assert getattr(L, n) is not None


def test_binding_covers_the_header_with_the_same_names(lib_path):
    assert sorted(dpd._SIGS) == _declared()
    for n in _declared():
        assert callable(getattr(dpd, n))
    dpd.load_library()


def test_no_gpu_means_a_loud_error():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dpd.DPDError) as e:
        dpd.dpd_create((10.0, 10.0, 12.0), 3.0, (25, 25, 25, 0), 4.5, 3.0, 1.0, 0.01, (0, 0, 0))
    assert e.value.code == dpd.DPD_ECUDA
