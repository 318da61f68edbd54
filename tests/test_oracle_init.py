"""Pins of the oracle's particle set-up from the phase field (Sec. II.C, reading R20).

* round(rho V) sites, uniform over the box (chi-square over unit cells).
* Maxwellian fluid velocities: mean exactly removed, variance kBT per component,
  normal (Kolmogorov-Smirnov), components uncorrelated.
* Classification by the phase field reproduces the geometry it encodes: in the
  planar channel field phi = tanh(d / (sqrt(2) eps)) every fluid site lies in the gap,
  every kept solid site within solid_layer of a wall, every removed site deeper --
  which pins phi_min = tanh(-solid_layer / (sqrt(2) eps)) (Eq. 14 read backwards).
* Same seed, same particles; another seed or system index, other particles.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1807_09896_gb300 import inputs

SQ2 = math.sqrt(2.0)


def _phi_min(layer, eps=0.5):
    return math.tanh(-layer / (SQ2 * eps))


def test_sites_fill_the_box_uniformly_without_a_phase_field():
    box = (10.0, 10.0, 10.0)
    out = oracle.init_particles(box, 3.0, 1.0, seed=4, phi_min=-1.0)
    assert out["n0"] == 3000 and len(out["pos"]) == 3000
    assert np.all(out["type"] == 0)
    p = out["pos"]
    assert p.min() >= 0.0 and np.all(p < np.asarray(box))
    counts = np.histogramdd(p, bins=(10, 10, 10), range=[(0, 10)] * 3)[0].ravel()
    chi2 = ((counts - 3.0) ** 2 / 3.0).sum()
    assert stats.chi2.sf(chi2, df=999) > 1e-3
    np.testing.assert_array_equal(out["site"], np.arange(3000))


def test_velocities_are_maxwellian_with_the_mean_removed():
    out = oracle.init_particles((12.0, 12.0, 12.0), 3.0, 0.7, seed=9, phi_min=-1.0)
    v = out["vel"]
    assert np.abs(v.mean(0)).max() < 1e-12
    var = v.var(0)
    n = len(v)
    assert np.all(np.abs(var / 0.7 - 1.0) < 5 * math.sqrt(2.0 / n))
    for a in range(3):
        assert stats.kstest(v[:, a] / math.sqrt(0.7), "norm").pvalue > 1e-3
    c = np.corrcoef(v.T)
    assert np.abs(c - np.eye(3)).max() < 5 / math.sqrt(n)


@pytest.mark.parametrize("layer", [0.5, 1.0])
def test_classification_follows_the_distance_the_phase_field_encodes(layer):
    H = 6.0
    w = inputs.channel(8.0, 7.0, H, seed=0)  # walls at z = 0 and z = H, box height H + 2
    field = oracle.Field(w.phi, w.h)
    out = oracle.init_particles(w.box, 3.0, 1.0, seed=5, phi_min=_phi_min(layer), field=field)
    Lz = w.box[2]
    z = out["pos"][:, 2]
    # signed distance to the nearer wall: positive in the gap, negative in the solid
    d = np.where(z <= H, np.minimum(z, H - z), -np.minimum(z - H, Lz - z))
    fluid, solid = out["type"] == 0, out["type"] == 1
    tol = 0.02  # trilinear interpolation of the tanh profile on a 0.25 grid
    assert np.all(d[fluid] > -tol)
    assert np.all((d[solid] < tol) & (d[solid] > -layer - tol))
    # removed sites are the deeper ones
    removed = out["site_type"] == 2
    assert removed.any() == (layer < 1.0)
    # counts: fluid ~ H/Lz of the sites, solid ~ 2 layer / Lz
    n0 = out["n0"]
    for frac, expect in ((fluid.sum() / n0, H / Lz), (solid.sum() / n0, 2 * min(layer, 1.0) / Lz)):
        assert abs(frac - expect) < 5 * math.sqrt(expect * (1 - expect) / n0)
    # every kept site's phase field agrees with its class
    phi = out["site_phi"][out["site"]]
    assert np.all(phi[fluid] >= 0.0) and np.all((phi[solid] < 0.0) & (phi[solid] > _phi_min(layer)))


def test_same_seed_same_particles_other_seed_or_system_other_particles():
    a = oracle.init_particles((6.0, 5.0, 4.0), 3.0, 1.0, seed=11, phi_min=-1.0)
    b = oracle.init_particles((6.0, 5.0, 4.0), 3.0, 1.0, seed=11, phi_min=-1.0)
    c = oracle.init_particles((6.0, 5.0, 4.0), 3.0, 1.0, seed=12, phi_min=-1.0)
    d = oracle.init_particles((6.0, 5.0, 4.0), 3.0, 1.0, seed=11, phi_min=-1.0, sys=1)
    np.testing.assert_array_equal(a["pos"], b["pos"])
    np.testing.assert_array_equal(a["vel"], b["vel"])
    assert not np.allclose(a["pos"], c["pos"]) and not np.allclose(a["pos"], d["pos"])
