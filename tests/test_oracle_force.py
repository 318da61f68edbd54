"""Pins of the oracle's neighbour search and pair force (Sec. II.A, Eqs. 2-10).

* the cell-list neighbour set equals the all-pairs set, and both equal a numpy
  all-pairs search with the minimum image (cutoff r < r_c = 1, Sec. II.A);
* conservative part (Eqs. 4-5): the force is minus the gradient of the pair
  energy U = sum a_ij (1 - r)^2 / 2, checked by central differences, with
  a_ff != a_fs so that the a_ij lookup is pinned too;
* dissipative part (Eq. 6): Galilean invariance, zero response to motion
  perpendicular to the line of centres, linearity in gamma, and a strictly
  negative dissipated power;
* random part (Eq. 7 with the 1/sqrt(dt) of the discrete scheme): the variance of
  the pair force along the line of centres over independent steps is
  sigma^2 w_R^2 / dt;
* all parts: f_ij = -f_ji, so the total force of a periodic fluid is zero
  (momentum conservation, Sec. II.A); axis permutation covariance.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1807_09896_gb300 import inputs


def _np_pairs(pos, box):
    pos = np.asarray(pos, np.float64)
    L = np.asarray(box, np.float64)
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.round(d / L)
    r2 = (d * d).sum(-1)
    i, j = np.nonzero(np.triu(r2 < 1.0, k=1))
    return np.stack([i, j], axis=1)


@pytest.mark.parametrize("box,seed", [((3.0, 3.0, 3.0), 0), ((4.0, 3.0, 5.0), 1),
                                      ((5.0, 5.0, 5.0), 2), ((3.5, 4.25, 6.0), 3)])
def test_cell_list_pairs_equal_all_pairs(box, seed):
    rng = np.random.default_rng(seed)
    n = int(3 * np.prod(box))
    pos = rng.uniform(0, 1, (n, 3)) * np.asarray(box)
    brute = oracle.pairs(pos, box, method=0)
    cells = oracle.pairs(pos, box, method=1)
    ref = _np_pairs(pos, box)
    assert len(brute) > 0
    np.testing.assert_array_equal(brute, cells)
    np.testing.assert_array_equal(brute, ref)


def _energy(pos, types, box, a_ff, a_fs):
    L = np.asarray(box)
    U = 0.0
    for i, j in _np_pairs(pos, box):
        if types[i] and types[j]:
            continue
        d = pos[i] - pos[j]
        d -= L * np.round(d / L)
        r = math.sqrt(d @ d)
        a = a_ff if (types[i] == 0 and types[j] == 0) else a_fs
        U += 0.5 * a * (1.0 - r) ** 2
    return U


def test_conservative_force_is_minus_energy_gradient():
    w = inputs.channel(3.0, 3.0, 3.0, seed=4)
    p = oracle.Params(box=w.box, a_ff=25.0, a_fs=40.0, gamma=0.0, sigma=0.0)
    pos = w.pos.astype(np.float64)
    f = oracle.forces(pos, np.zeros_like(pos), w.id, w.type, p, step=0)
    eps = 1e-6
    rng = np.random.default_rng(0)
    fluid = np.nonzero(w.type == 0)[0]
    for i in rng.choice(fluid, size=12, replace=False):
        for a in range(3):
            pp = pos.copy(); pp[i, a] += eps
            pm = pos.copy(); pm[i, a] -= eps
            g = (_energy(pp, w.type, w.box, 25.0, 40.0) - _energy(pm, w.type, w.box, 25.0, 40.0)) / (2 * eps)
            assert abs(f[i, a] + g) < 1e-6 * max(1.0, abs(g)), (i, a, f[i, a], -g)
    assert np.all(f[w.type != 0] == 0.0)


def _bulk(seed=0, L=4.0):
    return inputs.bulk(L, seed=seed)


def test_dissipative_galilean_invariant_and_linear_in_gamma():
    w = _bulk(1)
    pos = w.pos.astype(np.float64)
    v = w.vel.astype(np.float64)
    p = oracle.Params(box=w.box, a_ff=0.0, gamma=4.5, sigma=0.0)
    f1 = oracle.forces(pos, v, w.id, w.type, p, 0)
    f2 = oracle.forces(pos, v + np.array([0.3, -1.2, 2.0]), w.id, w.type, p, 0)
    np.testing.assert_allclose(f2, f1, rtol=0, atol=1e-11 * np.abs(f1).max())
    p2 = oracle.Params(box=w.box, a_ff=0.0, gamma=9.0, sigma=0.0)
    f3 = oracle.forces(pos, v, w.id, w.type, p2, 0)
    np.testing.assert_allclose(f3, 2 * f1, rtol=1e-12, atol=1e-12)
    assert np.abs(f1).max() > 0.1


def test_dissipative_ignores_perpendicular_motion_and_dissipates():
    box = (4.0, 4.0, 4.0)
    pos = np.array([[1.0, 1.0, 1.0], [1.6, 1.0, 1.0]])
    ids = np.array([0, 1], np.int32)
    types = np.zeros(2, np.uint8)
    p = oracle.Params(box=box, a_ff=0.0, gamma=4.5, sigma=0.0)
    v_perp = np.array([[0.0, 1.0, -0.5], [0.0, -1.0, 0.25]])
    assert np.abs(oracle.forces(pos, v_perp, ids, types, p, 0)).max() == 0.0
    v_close = np.array([[1.0, 0.0, 0.0], [-1.0, 0.0, 0.0]])  # approaching along x
    f = oracle.forces(pos, v_close, ids, types, p, 0)
    assert f[0, 0] < 0.0 < f[1, 0]  # friction opposes the approach
    w = _bulk(2)
    v = w.vel.astype(np.float64)
    fb = oracle.forces(w.pos.astype(np.float64), v, w.id, w.type, p, 0)
    assert (fb * v).sum() < 0.0


def test_random_force_variance_along_line_of_centres():
    box = (4.0, 4.0, 4.0)
    r = 0.4
    pos = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
    ids = np.array([3, 11], np.int32)
    types = np.zeros(2, np.uint8)
    dt, sigma = 0.01, 3.0
    p = oracle.Params(box=box, a_ff=0.0, gamma=0.0, sigma=sigma, dt=dt, seed=5)
    v = np.zeros((2, 3))
    samples = np.array([oracle.forces(pos, v, ids, types, p, s)[0] for s in range(20000)])
    assert np.all(samples[:, 1:] == 0.0)
    fx = samples[:, 0]
    expect = sigma ** 2 * (1 - r) ** 2 / dt
    n = len(fx)
    assert abs(fx.mean()) < 5 * math.sqrt(expect / n)
    assert abs(fx.var() / expect - 1.0) < 5 * math.sqrt(2.0 / n)


@pytest.mark.parametrize("seed", [0, 1])
def test_total_force_vanishes_in_periodic_fluid(seed):
    w = _bulk(seed, L=5.0)
    p = oracle.Params(box=w.box, seed=seed)
    f = oracle.forces(w.pos.astype(np.float64), w.vel.astype(np.float64), w.id, w.type, p, 17)
    assert np.abs(f.sum(axis=0)).max() < 1e-12 * np.abs(f).sum()
    assert np.abs(f).max() > 10.0


def test_axis_permutation_covariance():
    w = _bulk(3, L=4.0)
    pos = w.pos.astype(np.float64)
    v = w.vel.astype(np.float64)
    p = oracle.Params(box=w.box, seed=9)
    f = oracle.forces(pos, v, w.id, w.type, p, 4)
    perm = [1, 2, 0]
    fp = oracle.forces(pos[:, perm], v[:, perm], w.id, w.type, p, 4)
    np.testing.assert_allclose(fp, f[:, perm], rtol=1e-12, atol=1e-12)


def test_brute_and_cell_forces_agree():
    w = inputs.channel(4.0, 3.0, 3.0, seed=6)
    p = oracle.Params(box=w.box, seed=3)
    pos = w.pos.astype(np.float64)
    v = w.vel.astype(np.float64)
    f0 = oracle.forces(pos, v, w.id, w.type, p, 2, method=0)
    f1 = oracle.forces(pos, v, w.id, w.type, p, 2, method=1)
    np.testing.assert_allclose(f0, f1, rtol=1e-12, atol=1e-10)
