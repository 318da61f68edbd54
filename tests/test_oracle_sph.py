"""Pins of the attractive/repulsive pair force of Sec. IV (Eqs. 22-24) in the oracle.

* Eq. 23's alpha_D normalises the smoothing function: its integral over 1-, 2- and
  3-D space is 1 (this fixes alpha_D = 2/3, 10/(7 pi), 1/pi and h = r0 / 2).
* The cubic spline is C^2: W and dW/dr are continuous at v = 1 and vanish with the
  second derivative at the edge of the support v = 2 (r = r0).
* dW/dr is the derivative of W (central differences).
* The conservative pair force is minus the derivative of the pair energy of Eq. 22
  along the separation (reading R19): repulsive at short range (the S^r term wins),
  attractive further out (the S^a term), zero beyond r0^a.
* Fluid-solid pairs use their own strengths: the paper's doubled values give twice
  the fluid-fluid force at every separation.
"""
import math

import numpy as np
import pytest

import oracle


def _integral(D, r0, n=200001):
    r = np.linspace(0.0, r0, n)
    W = np.array([oracle.sph_W(x, r0, D) for x in r])
    shell = {1: 2.0 * np.ones_like(r), 2: 2 * math.pi * r, 3: 4 * math.pi * r * r}[D]
    trapezoid = getattr(np, "trapezoid", None) or np.trapz
    return trapezoid(W * shell, r)


@pytest.mark.parametrize("D", [1, 2, 3])
@pytest.mark.parametrize("r0", [0.73, 1.0])
def test_smoothing_function_is_normalised(D, r0):
    assert abs(_integral(D, r0, n=20001) - 1.0) < 1e-6


@pytest.mark.parametrize("D", [2, 3])
def test_spline_is_smooth_at_its_knots_and_vanishes_at_the_support_edge(D):
    r0 = 0.73
    h = r0 / 2
    e = 1e-7
    for knot in (h, r0):
        assert abs(oracle.sph_W(knot - e, r0, D) - oracle.sph_W(knot + e, r0, D)) < 1e-5
        assert abs(oracle.sph_dWdr(knot - e, r0, D) - oracle.sph_dWdr(knot + e, r0, D)) < 1e-4
    assert oracle.sph_W(r0, r0, D) == 0.0 and oracle.sph_dWdr(r0, r0, D) == 0.0
    assert oracle.sph_W(1.5 * r0, r0, D) == 0.0
    # second derivative continuous at v = 1 (from one-sided differences of dW/dr)
    d = 1e-5
    left = (oracle.sph_dWdr(h - d, r0, D) - oracle.sph_dWdr(h - 2 * d, r0, D)) / d
    right = (oracle.sph_dWdr(h + 2 * d, r0, D) - oracle.sph_dWdr(h + d, r0, D)) / d
    assert abs(left - right) < 1e-2 * abs(left)


@pytest.mark.parametrize("D", [2, 3])
def test_dWdr_is_the_derivative_of_W(D):
    r0 = 1.0
    d = 1e-6
    for r in np.linspace(0.05, 0.95, 19):
        fd = (oracle.sph_W(r + d, r0, D) - oracle.sph_W(r - d, r0, D)) / (2 * d)
        assert abs(oracle.sph_dWdr(r, r0, D) - fd) < 1e-6 * max(1.0, abs(fd))


def _pair_force(p, r, solid=False, direction=(0.6, 0.0, 0.8)):
    e = np.asarray(direction)
    pos = np.array([[2.0, 2.0, 2.0], [2.0, 2.0, 2.0] - r * e])
    types = np.array([0, 1 if solid else 0], np.uint8)
    f = oracle.forces(pos, np.zeros((2, 3)), np.arange(2, dtype=np.int32), types, p, 0)
    return f[0], e


@pytest.mark.parametrize("D", [2, 3])
def test_pair_force_is_minus_the_energy_gradient(D):
    p = oracle.Params(box=(6.0, 6.0, 6.0), gamma=0.0, sigma=0.0, force_law=1, sph_dim=D)
    d = 1e-6
    signs = []
    for r in np.linspace(0.05, 0.99, 30):
        f, e = _pair_force(p, r)
        minus_dE = -(oracle.sph_energy(p, r + d) - oracle.sph_energy(p, r - d)) / (2 * d)
        np.testing.assert_allclose(f, minus_dE * e, atol=1e-5 * max(1.0, abs(minus_dE)))
        signs.append(np.sign(f @ e))
    # repulsive (along r_i - r_j) at short range, attractive further out
    assert signs[0] > 0 and signs[-2] < 0
    f, _ = _pair_force(p, 1.0 - 1e-9)
    assert np.abs(f).max() < 1e-6  # nothing beyond r0^a = 1


def test_fluid_solid_pairs_feel_the_doubled_strengths():
    p = oracle.Params(box=(6.0, 6.0, 6.0), gamma=0.0, sigma=0.0, force_law=1)
    for r in (0.1, 0.3, 0.5, 0.8):
        f_ff, _ = _pair_force(p, r)
        f_fs, _ = _pair_force(p, r, solid=True)
        np.testing.assert_allclose(f_fs, 2.0 * f_ff, rtol=1e-12)


def test_force_law_0_is_unchanged_by_the_spline_parameters():
    a = oracle.Params(box=(6.0, 6.0, 6.0), gamma=0.0, sigma=0.0)
    b = oracle.Params(box=(6.0, 6.0, 6.0), gamma=0.0, sigma=0.0, S_r_ff=1.0, r0_r=0.5)
    for r in (0.2, 0.7):
        np.testing.assert_array_equal(_pair_force(a, r)[0], _pair_force(b, r)[0])
        np.testing.assert_allclose(_pair_force(a, r)[0] @ np.array([0.6, 0, 0.8]), 25.0 * (1 - r))
