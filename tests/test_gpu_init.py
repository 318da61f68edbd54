"""GPU particle set-up from the phase field (dpd_init_particles, Sec. II.C) against
the oracle's, through the C ABI.

Both draw the same Philox sites.  A GPU position is the binary32 rounding of the
exact product u L, so it equals the oracle's FP64 position rounded to binary32 bit
for bit; particles are matched on that.  Classes agree except for sites whose phase
field lies within 1e-5 of a threshold (binary32 interpolation); velocities agree to
binary32 rounding (< 2e-5).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1807_09896_gb300 import dpd, inputs
from parity_helpers import gpu_state

pytestmark = pytest.mark.gpu
AMBIGUOUS = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_09896_gb300 import _build

    _build.build()


def _gpu_init(w, seed, layer, kBT=1.0, rho=3.0, sys=0, field=True):
    s = dpd.System(w.box, kBT=kBT, rho=rho, system=sys)
    if field:
        dpd.dpd_set_phase_field(s.h, w.phi, w.h)
    s.init_particles(seed, layer)
    return s


def _compare(w, seed, layer, kBT=1.0, rho=3.0, sys=0, field=True):
    s = _gpu_init(w, seed, layer, kBT, rho, sys, field)
    pos, vel, _, types = gpu_state(s)
    phi_min = math.tanh(-layer / (math.sqrt(2.0) * 0.5))
    ref = oracle.init_particles(w.box, rho, kBT, seed, phi_min,
                                oracle.Field(w.phi, w.h) if field else None, sys=sys)
    # sites whose class depends on binary32 rounding of the interpolated phase field
    sp = ref["site_phi"]
    amb_sites = (np.abs(sp) < AMBIGUOUS) | (np.abs(sp - phi_min) < AMBIGUOUS)
    index = {tuple(p): k for k, p in enumerate(ref["pos"].astype(np.float32))}
    matched = np.array([index.get(tuple(p), -1) for p in pos])
    unmatched_gpu = matched < 0
    # a GPU particle without an oracle partner must sit on an ambiguous site
    if unmatched_gpu.any():
        assert unmatched_gpu.sum() <= amb_sites.sum()
    m = matched[~unmatched_gpu]
    np.testing.assert_array_equal(types[~unmatched_gpu], ref["type"][m])
    assert len(ref["pos"]) - len(m) <= amb_sites.sum()
    # ids follow the site order
    assert np.all(np.diff(ref["site"][m]) > 0)
    dv = np.abs(vel[~unmatched_gpu].astype(np.float64) - ref["vel"][m])
    assert dv.max() < 2e-5, dv.max()
    nf = int((types == 0).sum())
    if nf:
        assert np.abs(vel[types == 0].astype(np.float64).mean(0)).max() < 1e-6
    return s, len(pos), nf


@pytest.mark.parametrize("layer", [0.5, 1.0])
def test_channel_set_up_matches_the_oracle(layer):
    w = inputs.channel(8.0, 7.0, 6.0, seed=0)
    s, n, nf = _compare(w, seed=21, layer=layer)
    assert 0 < nf < n
    s.step(20)  # the set-up state steps without error
    s.close()


def test_sphere_pack_and_bulk_set_up_match_the_oracle():
    w = inputs.sphere_pack(12.0, 3, 2.0, 3.0, seed=5)
    s, n, nf = _compare(w, seed=3, layer=1.0, kBT=0.5, sys=2)
    assert nf < n
    s.close()
    b = inputs.bulk((5.0, 6.0, 7.0), seed=1)
    s, n, nf = _compare(b, seed=8, layer=1.0, field=False)
    assert n == nf == round(3.0 * 5 * 6 * 7)
    s.close()


def test_full_size_channel_set_up_matches_the_oracle():
    w = inputs.channel(80.0, 64.0, 64.0, seed=0)
    s, n, nf = _compare(w, seed=0, layer=1.0)
    assert abs(nf - 3.0 * 80 * 64 * 64) < 5 * math.sqrt(3.0 * 80 * 64 * 64)
    s.close()


def test_set_up_is_deterministic_and_rejects_a_negative_layer():
    w = inputs.channel(8.0, 7.0, 6.0, seed=0)
    a = _gpu_init(w, 5, 1.0)
    b = _gpu_init(w, 5, 1.0)
    for x, y in zip(gpu_state(a), gpu_state(b)):
        np.testing.assert_array_equal(x, y)
    with pytest.raises(dpd.DPDError):
        a.init_particles(5, -1.0)
    a.close()
    b.close()
