"""The library's device Philox4x32-10 against cuRAND's (the vendor library's raw
Philox4x32-10 on the same counter and key), word for word, on random and edge-case
inputs including the counters the pair noise and the particle set-up use."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def helper():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, "philox_curand_check.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                    "-Xcompiler", "-fPIC", os.path.join(HERE, "philox_curand_check.cu"), "-o", so],
                   check=True)
    lib = ctypes.CDLL(so)
    lib.philox_both.restype = ctypes.c_int
    return lib


def _run(lib, ctr, key):
    ctr = np.ascontiguousarray(ctr, np.uint32)
    key = np.ascontiguousarray(key, np.uint32)
    n = len(ctr)
    ours = np.zeros((n, 4), np.uint32)
    theirs = np.zeros((n, 4), np.uint32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.philox_both(p(ctr), p(key), n, p(ours), p(theirs)) == 0
    return ours, theirs


def test_device_philox_equals_curand(helper):
    rng = np.random.default_rng(0)
    n = 1 << 16
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    # edge cases: zeros, all ones, the set-up counters, a typical pair-noise counter
    ctr[:6] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [7, 0xFFFFFFFF, 0xFFFFFFFE, 0],
               [7, 0xFFFFFFFF, 0xFFFFFFFD, 3], [12, 345, 1000, 0], [0, 1, 0, 1]]
    key[:6] = [[0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [1, 0], [1, 0], [0, 0], [0x12345678, 0x9ABCDEF0]]
    ours, theirs = _run(helper, ctr, key)
    np.testing.assert_array_equal(ours, theirs)
