"""The allocation-free profile entry point, for callers that cannot allocate device
memory (a framework that owns all device memory through its own pool, a process
under a hard memory cap, a latency-bound loop where an allocation would stall the
device).  It must give the same sums as the handle-based dpd_velocity_profile on
the same particles, on consecutive calls (its fixed accumulators are shared by
every call and must be cleared each time).

This file is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1807_09896_gb300 import dpd, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_09896_gb300 import _build

    _build.build()
    return torch


def _device_state(torch, s, n):
    pos = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    vel = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    typ = torch.empty((n,), dtype=torch.uint8, device="cuda")
    dpd.dpd_get_state(s.h, pos, vel, None, None, typ, where=dpd.DPD_DEVICE)
    torch.cuda.synchronize()
    return pos, vel, typ


def test_noalloc_profile_matches_the_handle_profile_on_consecutive_calls(torch_cuda):
    torch = torch_cuda
    w = inputs.channel(8.0, 6.0, 6.0, seed=21)
    s = dpd.System.from_workload(w, g=(0.05, 0.0, 0.0), seed=4)
    s.step(12)
    pos, vel, typ = _device_state(torch, s, w.n)
    layouts = [(2, 24, 0.0, 6.0), (0, 16, 0.0, 8.0)]
    for call, (axis, nb, lo, hi) in enumerate(layouts):
        ref = s.profile(axis, nb, lo, hi, mode=1)  # the existing entry point
        out = np.full((nb, 5), np.nan)
        dpd.dpd_velocity_profile_noalloc(pos, vel, typ, w.n, axis, nb, lo, hi, out)
        np.testing.assert_array_equal(out[:, 0], ref[:, 0])  # counts: exact
        np.testing.assert_allclose(out[:, 1:], ref[:, 1:], rtol=1e-12, atol=1e-9)
        assert out[:, 0].sum() == w.n_fluid, call
    # a second call with the first layout again: nothing left over from the previous call
    axis, nb, lo, hi = layouts[0]
    ref = s.profile(axis, nb, lo, hi, mode=1)
    out_dev = torch.full((nb, 5), float("nan"), dtype=torch.float64, device="cuda")
    dpd.dpd_velocity_profile_noalloc(pos, vel, typ, w.n, axis, nb, lo, hi, out_dev,
                                     where=dpd.DPD_DEVICE)
    torch.cuda.synchronize()
    got = out_dev.cpu().numpy()
    np.testing.assert_array_equal(got[:, 0], ref[:, 0])
    np.testing.assert_allclose(got[:, 1:], ref[:, 1:], rtol=1e-12, atol=1e-9)
    s.close()


def test_noalloc_profile_rejects_more_bins_than_its_fixed_scratch(torch_cuda):
    torch = torch_cuda
    n = 8
    pos = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    vel = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    typ = torch.zeros((n,), dtype=torch.uint8, device="cuda")
    nb = dpd.NOALLOC_MAX_BINS + 1
    with pytest.raises(dpd.DPDError) as e:
        dpd.dpd_velocity_profile_noalloc(pos, vel, typ, n, 2, nb, 0.0, 1.0, np.zeros((nb, 5)))
    assert e.value.code == dpd.DPD_EINVAL
    assert "DPD_NOALLOC_MAX_BINS" in str(e.value)
