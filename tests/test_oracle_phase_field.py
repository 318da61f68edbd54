"""Pins of the FP64 phase-field relaxation oracle (Sec. II.B, Eqs. 13-15) to closed forms.

* A planar interface of any orientation with the profile of Eq. 14,
  tanh(d / (sqrt(2) eps)), is a steady state of both Eq. 13 and Eq. 15: the discrete
  right-hand side vanishes to second order in h / eps.  An oblique normal (1, 2, 2)/3
  exercises every mixed derivative.
* For a sphere with that profile in r, the curvature term of Eq. 15 cancels the
  whole curvature drift (rhs ~ 0), while Eq. 13 alone leaves exactly
  (2 / r) d phi / dr in scaled units (the Laplacian in spherical coordinates).
* Relaxing a step function: a planar step becomes the tanh profile; a sphere keeps
  its radius under Eq. 15 and shrinks by motion by mean curvature, R^2 = R0^2 - 4 t',
  under Eq. 13 (the sharp-interface limit of the Allen-Cahn equation).
"""
import numpy as np
import pytest

from oracle import phase_field as pf

SQ2 = np.sqrt(2.0)


def _grid(n, h):
    c = (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return c, x, y, z


def _inner(shape):
    m = np.zeros(shape, bool)
    m[1:-1, 1:-1, 1:-1] = True  # rolled differences wrap at the faces of a non-periodic field
    return m


def _planar_err(hp, curvature):
    eps = 1.0
    n = int(round(12 / hp))
    _, x, y, z = _grid(n, hp * eps)
    d = (x + 2 * y + 2 * z) / 3.0 - 6.3
    phi = np.tanh(d / (SQ2 * eps))
    r = pf.rhs(phi, hp * eps, eps, curvature)
    return np.abs(r[_inner(phi.shape)]).max()


@pytest.mark.parametrize("curvature", [True, False])
def test_oblique_planar_tanh_profile_is_steady_to_second_order(curvature):
    e1, e2 = _planar_err(0.5, curvature), _planar_err(0.25, curvature)
    assert e2 < 0.01
    assert e1 / e2 > 3.5  # second order: halving h divides the error by ~4


def _sphere(hp, R=4.0):
    eps = 1.0
    n = int(round(12 / hp))
    _, x, y, z = _grid(n, hp * eps)
    rr = np.sqrt((x - 6.0) ** 2 + (y - 6.0) ** 2 + (z - 6.0) ** 2)
    phi = np.tanh((R - rr) / (SQ2 * eps))
    dphi_dr = -1.0 / (SQ2 * eps) / np.cosh((R - rr) / (SQ2 * eps)) ** 2
    mask = _inner(phi.shape) & (rr > 1.0)
    return phi, hp * eps, eps, rr, dphi_dr, mask


def test_curvature_term_cancels_the_drift_of_a_sphere():
    errs = []
    for hp in (0.5, 0.25):
        phi, h, eps, rr, dphi, m = _sphere(hp)
        errs.append(np.abs(pf.rhs(phi, h, eps, True)[m]).max())
    assert errs[1] < 0.012 and errs[0] / errs[1] > 3.0


def test_without_curvature_term_a_sphere_feels_2_over_r_dphi_dr():
    errs = []
    for hp in (0.5, 0.25):
        phi, h, eps, rr, dphi, m = _sphere(hp)
        exact = (2.0 / rr) * dphi
        errs.append(np.abs(pf.rhs(phi, h, eps, False) - exact)[m].max())
        assert np.abs(exact[m]).max() > 0.3  # the drift itself is O(1)
    assert errs[1] < 0.007 and errs[0] / errs[1] > 3.0


def test_planar_step_relaxes_to_the_tanh_profile():
    eps, hp = 0.5, 0.5
    h = hp * eps
    n = 64
    c = (np.arange(n) + 0.5) * h
    L = n * h
    phi0 = np.where((c > L / 4) & (c < 3 * L / 4), 1.0, -1.0)
    phi0 = np.broadcast_to(phi0, (4, 4, n)).copy()
    out = pf.relax(phi0, h, eps, 500, 0.04, True)
    d = np.minimum(c - L / 4, 3 * L / 4 - c)  # signed distance to the nearer interface
    exact = np.tanh(d / (SQ2 * eps))
    assert np.abs(out - exact).max() < 0.02
    # x -> L/2 - x maps the step onto minus itself and the equation is odd in phi, so
    # the interface at L/4 stays put: phi(c_k) = -phi(L/2 - c_k)
    np.testing.assert_allclose(out[0, 0, :32], -out[0, 0, 31::-1], atol=1e-12)
    np.testing.assert_array_equal(out[0, 0], out[3, 2])  # no y, z dependence appears


def _ray_radius(phi, c, centre):
    """Zero crossing of phi along the +x ray through the centre, by linear interpolation."""
    i0 = len(c) // 2
    a = phi[i0, i0, :]
    k = np.where((a[:-1] > 0) & (a[1:] <= 0) & (c[:-1] > centre))[0][0]
    t = a[k] / (a[k] - a[k + 1])
    return c[k] + t * (c[k + 1] - c[k]) - centre


@pytest.mark.parametrize("curvature", [True, False])
def test_sphere_radius_is_kept_by_eq15_and_shrinks_by_mean_curvature_without_it(curvature):
    eps, hp, n = 0.5, 0.5, 48
    h = hp * eps
    c, x, y, z = _grid(n, h)
    centre = n * h / 2
    R0 = 7.0  # in units of eps
    rr = np.sqrt((x - centre) ** 2 + (y - centre) ** 2 + (z - centre) ** 2)
    phi = np.where(rr < R0 * eps, 1.0, -1.0)
    tp = 6.0
    out = pf.relax(phi, h, eps, 150, tp / 150, curvature)
    R = _ray_radius(out, c, centre) / eps
    if curvature:
        assert abs(R - R0) < 0.01
    else:
        assert abs(R - np.sqrt(R0 ** 2 - 4 * tp)) < 0.1
