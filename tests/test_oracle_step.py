"""Pins of the oracle's time step: integrator (Sec. II.A, ref. 35), phase-field
interpolation and bounce-back reflection (Sec. II.C, Eq. 17, Fig. 4), and the
profile sums (Sec. III.A).

* ballistic motion under the body force alone is exact: r = r0 + v0 t + g t^2/2;
* with only conservative forces and lambda = 1/2 the total energy error of the
  velocity-Verlet scheme is second order in dt (halving dt quarters it);
* the fluctuation-dissipation pair gamma = sigma^2 / 2 k_BT (Eq. 8) holds the
  kinetic temperature at k_BT (Sec. III.A: deviations measure integration error);
* trilinear interpolation returns node values and reproduces affine fields;
* a particle crossing a planar phi = 0 surface is put back at the mirror point of
  its would-be position (Fig. 4: phi_bb ~ -phi(t+dt)), with all velocity
  components reversed and no closing half-kick; a mirror point that is itself in
  the solid sends the particle back to r(t);
* no fluid particle ends a step at phi < 0 (Sec. II.C), frozen particles stay put.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1807_09896_gb300 import inputs


def _state(w, vel=None):
    s = oracle.State(w.pos.astype(np.float64), (w.vel if vel is None else vel).astype(np.float64),
                     np.zeros((w.n, 3)), w.id.copy(), w.type.copy())
    return s


def _field(w):
    return oracle.Field(w.phi, w.h)


def test_ballistic_motion_under_body_force_is_exact():
    w = inputs.bulk(4.0, seed=1)
    g = (0.3, -0.2, 0.05)
    p = oracle.Params(box=w.box, a_ff=0.0, gamma=0.0, sigma=0.0, g=g, dt=0.02)
    s = oracle.init_forces(_state(w), p)
    r0, v0 = s.pos.copy(), s.vel.copy()
    for _ in range(25):
        s = oracle.step(s, p, _field(w))
    t = 25 * p.dt
    expect = r0 + v0 * t + 0.5 * np.asarray(g) * t * t
    L = np.asarray(w.box)
    d = s.pos - expect
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-12
    np.testing.assert_allclose(s.vel, v0 + np.asarray(g) * t, rtol=0, atol=1e-13)


def _energy(s, p):
    ke = 0.5 * (s.vel ** 2).sum()
    pairs = oracle.pairs(s.pos, p.box, method=1)
    L = np.asarray(p.box)
    d = s.pos[pairs[:, 0]] - s.pos[pairs[:, 1]]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(1))
    return ke + (0.5 * p.a_ff * (1 - r) ** 2).sum()


def _energy_error(dt, T=1.0):
    w = inputs.bulk(4.0, seed=2)
    p = oracle.Params(box=w.box, a_ff=25.0, gamma=0.0, sigma=0.0, dt=dt, lam=0.5)
    s = oracle.init_forces(_state(w), p)
    e0 = _energy(s, p)
    err = 0.0
    for _ in range(int(round(T / dt))):
        s = oracle.step(s, p, _field(w))
        err = max(err, abs(_energy(s, p) - e0))
    return err / e0


def test_velocity_verlet_energy_error_is_second_order():
    e1 = _energy_error(0.02)
    e2 = _energy_error(0.01)
    assert e1 < 1e-2
    assert 3.0 < e1 / e2 < 5.5, (e1, e2)


@pytest.mark.parametrize("kBT", [1.0, 0.5])
def test_fluctuation_dissipation_holds_temperature(kBT):
    w = inputs.bulk(6.0, seed=3, kBT=kBT)
    gamma = 4.5
    sigma = math.sqrt(2.0 * gamma * kBT)  # Eq. 8
    p = oracle.Params(box=w.box, a_ff=25.0, gamma=gamma, sigma=sigma, kBT=kBT, dt=0.01,
                      lam=0.65, seed=11)
    s = oracle.init_forces(_state(w), p)
    temps = []
    # the random start stores excess conservative energy; let the thermostat
    # remove it (about 5 time units) before sampling
    for k in range(2000):
        s = oracle.step(s, p, _field(w))
        if k >= 600:
            v = s.vel
            temps.append(((v - v.mean(0)) ** 2).sum() / (3 * (len(v) - 1)))
    T = float(np.mean(temps))
    assert abs(T / kBT - 1.0) < 0.03, T


def test_interpolation_nodes_and_affine_fields():
    h = 0.25
    nx, ny, nz = 12, 16, 20
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    grid = (0.5 * i * h - 0.25 * j * h + 0.125 * k * h + 0.1).astype(np.float32)
    f = oracle.Field(grid, h)
    rng = np.random.default_rng(0)
    nodes = np.stack([rng.integers(0, nx, 20), rng.integers(0, ny, 20), rng.integers(0, nz, 20)], 1)
    vals = oracle.phi_at(f, nodes * h)
    np.testing.assert_array_equal(vals, grid[nodes[:, 2], nodes[:, 1], nodes[:, 0]].astype(np.float64))
    # interior points (no periodic wrap between the corner nodes)
    pts = rng.uniform(0, 1, (50, 3)) * (np.array([nx, ny, nz]) - 1) * h
    expect = 0.5 * pts[:, 0] - 0.25 * pts[:, 1] + 0.125 * pts[:, 2] + 0.1
    np.testing.assert_allclose(oracle.phi_at(f, pts), expect, rtol=0, atol=2e-6)
    # periodicity
    L = np.array([nx, ny, nz]) * h
    np.testing.assert_allclose(oracle.phi_at(f, pts + L), oracle.phi_at(f, pts), atol=1e-12)
    np.testing.assert_allclose(oracle.phi_at(f, pts - 2 * L), oracle.phi_at(f, pts), atol=1e-12)


def _lone_particle(w, r0, v0):
    """One fluid particle in an otherwise empty copy of workload w."""
    pos = np.array([r0], np.float64)
    vel = np.array([v0], np.float64)
    return oracle.State(pos, vel, np.zeros((1, 3)), np.array([0], np.int32), np.zeros(1, np.uint8))


def test_bounce_back_lands_on_mirror_point_of_planar_wall():
    w = inputs.channel(3.0, 3.0, 3.0, seed=0)
    f = _field(w)
    p = oracle.Params(box=w.box, a_ff=0.0, gamma=0.0, sigma=0.0, dt=0.01)
    r0 = np.array([1.1, 1.3, 0.03])
    v0 = np.array([1.0, -2.0, -4.0])
    s = oracle.init_forces(_lone_particle(w, r0, v0), p)
    s1, refl = oracle.step(s, p, f, return_reflected=True)
    assert refl[0] and s1.stats["reflections"] == 1 and s1.stats["fallbacks"] == 0
    r1 = r0 + v0 * p.dt                  # would-be position, z = -0.01 (in the solid)
    # mirror of z = -0.01 about the phi = 0 plane z = 0 (Fig. 4, phi_bb ~ -phi(t+dt))
    assert abs(s1.pos[0, 2] - 0.01) < 1e-4
    # the reflected point moves back along the displacement: r_bb = r1 - 2 s dr, 0 < s < 1
    back = r1 - s1.pos[0]
    dr = v0 * p.dt
    sfrac = back[2] / (2 * dr[2])
    assert 0.0 < sfrac < 1.0
    np.testing.assert_allclose(back, 2 * sfrac * dr, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(s1.vel[0], -v0)  # bounce-back: all components reversed
    phi_new = oracle.phi_at(f, r1)[0]
    phi_bb = oracle.phi_at(f, s1.pos[0])[0]
    assert phi_new < 0 < phi_bb
    assert abs(phi_bb + phi_new) < 1e-3 * abs(phi_new)


def test_reflected_particle_skips_closing_half_kick():
    w = inputs.channel(3.0, 3.0, 3.0, seed=0)
    p = oracle.Params(box=w.box, a_ff=0.0, gamma=0.0, sigma=0.0, dt=0.01, g=(0.5, 0.0, 0.0))
    pos = np.array([[1.0, 1.0, 0.02], [1.0, 2.0, 1.5]])
    vel = np.array([[0.2, 0.1, -3.0], [0.2, 0.1, -3.0]])
    s = oracle.State(pos, vel, np.zeros((2, 3)), np.array([0, 1], np.int32), np.zeros(2, np.uint8))
    s = oracle.init_forces(s, p)
    s1, refl = oracle.step(s, p, _field(w), return_reflected=True)
    assert refl.tolist() == [True, False]
    np.testing.assert_array_equal(s1.vel[0], -vel[0])
    np.testing.assert_allclose(s1.vel[1], vel[1] + np.array([0.5, 0, 0]) * p.dt, atol=1e-15)


def test_mirror_point_inside_solid_falls_back_to_start():
    # a fluid film 1.0 < z < 1.2 between two solids, grid spacing 0.05
    box = (3.0, 3.0, 3.0)
    h = 0.05
    n = 60
    z = np.arange(n) * h
    d = np.minimum(z - 1.0, 1.2 - z)
    phi_z = np.tanh(d / (math.sqrt(2) * 0.5)).astype(np.float32)
    grid = np.broadcast_to(phi_z[:, None, None], (n, n, n)).astype(np.float32).copy()
    f = oracle.Field(grid, h)
    p = oracle.Params(box=box, a_ff=0.0, gamma=0.0, sigma=0.0, dt=0.01)
    r0 = np.array([1.0, 1.0, 1.19])
    v0 = np.array([0.0, 0.0, 25.0])  # would land at z = 1.44, mirror ~0.96 is solid
    s = oracle.State(np.array([r0]), np.array([v0]), np.zeros((1, 3)), np.array([0], np.int32),
                     np.zeros(1, np.uint8))
    s = oracle.init_forces(s, p)
    s1 = oracle.step(s, p, f)
    assert s1.stats == {"reflections": 1, "fallbacks": 1}
    np.testing.assert_array_equal(s1.pos[0], r0)
    np.testing.assert_array_equal(s1.vel[0], -v0)


def test_no_fluid_particle_ends_a_step_inside_the_solid():
    w = inputs.channel(5.0, 5.0, 4.0, seed=5)
    p = oracle.Params(box=w.box, g=(0.05, 0.0, 0.0), seed=2)
    f = _field(w)
    s = oracle.init_forces(_state(w), p)
    solid = w.type != 0
    spos = s.pos[solid].copy()
    fluid = ~solid
    for _ in range(300):
        s = oracle.step(s, p, f)
        assert oracle.phi_at(f, s.pos[fluid]).min() >= 0.0
    assert s.stats["reflections"] > 0
    np.testing.assert_array_equal(s.pos[solid], spos)
    assert np.all(s.vel[solid] == 0) and np.all(s.frc[solid] == 0)


def test_profile_counts_and_sums_at_bin_centres():
    nbins, lo, hi = 8, 0.0, 4.0
    centres = lo + (np.arange(nbins) + 0.5) * (hi - lo) / nbins
    reps = np.arange(1, nbins + 1)
    z = np.repeat(centres, reps)
    pos = np.stack([np.full_like(z, 0.5), np.full_like(z, 0.5), z], 1).astype(np.float32)
    vel = np.tile([[0.5, -1.0, 2.0]], (len(z), 1))
    types = np.zeros(len(z), np.uint8)
    types[0] = 1  # a solid particle is never counted
    out = oracle.profile(pos, vel, types, 2, nbins, lo, hi)
    counts = reps.astype(float)
    counts[0] -= 1
    np.testing.assert_array_equal(out[:, 0], counts)
    np.testing.assert_array_equal(out[:, 1], 0.5 * counts)
    np.testing.assert_array_equal(out[:, 2], -1.0 * counts)
    np.testing.assert_array_equal(out[:, 3], 2.0 * counts)
    np.testing.assert_array_equal(out[:, 4], 5.25 * counts)


def test_moving_wall_translates_the_solid_and_reflects_with_its_velocity():
    """Sec. II.C: at a wall moving with v_wall the bounce-back velocity is
    2 v_wall - v(t); the solid itself (its frozen particles) moves at v_wall."""
    w = inputs.channel(4.0, 3.0, 3.0, seed=2)
    vw = (0.5, -0.25, 0.0)
    p = oracle.Params(box=w.box, a_ff=0.0, a_fs=0.0, gamma=0.0, sigma=0.0, dt=0.01, v_wall=vw)
    pos = np.array([[1.0, 1.0, 0.02], [2.0, 1.5, 4.5]])  # a fluid particle, a solid one
    vel = np.array([[0.2, 0.1, -3.0], [0.0, 0.0, 0.0]])
    s = oracle.State(pos, vel, np.zeros((2, 3)), np.array([0, 1], np.int32),
                     np.array([0, 1], np.uint8))
    s = oracle.init_forces(s, p)
    s1, refl = oracle.step(s, p, _field(w), return_reflected=True)
    assert refl.tolist() == [True, False]
    np.testing.assert_allclose(s1.vel[0], 2 * np.asarray(vw) - vel[0], atol=1e-15)
    np.testing.assert_allclose(s1.pos[1], pos[1] + p.dt * np.asarray(vw), atol=1e-15)


def test_couette_walls_slide_oppositely_and_reflect_with_their_own_velocity():
    """Plane Couette walls (Sec. II.C moving walls, reading R18): the wall at z = H
    slides at +U and the one at z = 0 at -U, from the field v_w = (z - H/2) 2U/H.
    Frozen particles at either surface move with their wall; a particle bouncing off
    a wall leaves with 2 v_w - v of that wall (crossing point within ~0.01 of it)."""
    H, U = 3.0, 0.6
    w = inputs.channel(4.0, 3.0, H, seed=2)  # box z: fluid (0, H), solids up to H + 1, wrap at H + 2
    p = oracle.Params(box=w.box, a_ff=0.0, a_fs=0.0, gamma=0.0, sigma=0.0, dt=0.01,
                      shear=(2 * U / H, 0.0, 0.0), shear_axis=2, shear_ref=H / 2)
    pos = np.array([[1.0, 1.0, 0.02], [2.0, 1.0, H - 0.02],   # fluid heading into each wall
                    [1.5, 1.5, H], [2.5, 1.5, 0.0], [0.5, 0.5, H + 1.5]])  # solids
    vel = np.array([[0.2, 0.1, -3.0], [0.2, 0.1, 3.0], [0, 0, 0], [0, 0, 0], [0, 0, 0]], float)
    types = np.array([0, 0, 1, 1, 1], np.uint8)
    s = oracle.State(pos, vel, np.zeros((5, 3)), np.arange(5, dtype=np.int32), types)
    s = oracle.init_forces(s, p)
    s1, refl, vw = oracle.step(s, p, _field(w), return_reflected=True, return_wall_velocity=True)
    assert refl.tolist() == [True, True, False, False, False]
    np.testing.assert_allclose(s1.vel[0], [-2 * U - 0.2, -0.1, 3.0], atol=0.01)  # lower wall: -U
    np.testing.assert_allclose(s1.vel[1], [2 * U - 0.2, -0.1, -3.0], atol=0.01)  # upper wall: +U
    np.testing.assert_allclose(s1.vel[:2], 2 * vw[:2] - vel[:2], atol=1e-15)
    # solids: the upper surface moves at +U, the lower at -U, the layer between them
    # (z = H + 1.5, i.e. 0.5 below the lower surface through the wrap) at -U (1 + 1/H)
    np.testing.assert_allclose(vw[2:, 0], [U, -U, -U * (1 + 1.0 / H)], atol=1e-12)
    np.testing.assert_allclose(s1.pos[2:, 0], pos[2:, 0] + p.dt * vw[2:, 0], atol=1e-15)
    np.testing.assert_array_equal(s1.pos[2:, 1:], pos[2:, 1:])


def test_couette_walls_drag_nearby_fluid_along_their_own_velocity():
    """Frozen particles enter the dissipative force (Eq. 6) with the velocity of their
    own wall (reading R18): a fluid particle at rest near the upper wall (+U) is
    dragged towards +x, its mirror image near the lower wall (-U) equally towards -x,
    and with resting walls neither feels anything."""
    H, U = 3.0, 0.6
    w = inputs.channel(4.0, 3.0, H, seed=2)
    pos = np.array([[1.0, 1.0, H - 0.3], [1.3, 1.0, H + 0.3],       # near the upper wall
                    [1.0, 2.0, 0.3], [1.3, 2.0, H + 2 - 0.3]])      # mirror, through the wrap
    types = np.array([0, 1, 0, 1], np.uint8)
    ids = np.arange(4, dtype=np.int32)
    out = []
    for shear in ((2 * U / H, 0.0, 0.0), (0.0, 0.0, 0.0)):
        p = oracle.Params(box=w.box, a_ff=0.0, a_fs=0.0, gamma=4.5, sigma=0.0, dt=0.01,
                          shear=shear, shear_axis=2, shear_ref=H / 2)
        out.append(oracle.forces(pos, np.zeros((4, 3)), ids, types, p, 0))
    f, f0 = out
    assert f[0, 0] > 0 and f[2, 0] < 0
    np.testing.assert_allclose(f[2, 0], -f[0, 0], rtol=1e-12)
    # mirroring z flips f_z and reversing the wall velocity flips the dissipative
    # force: together f_z is unchanged
    np.testing.assert_allclose(f[2, 2], f[0, 2], rtol=1e-12)
    np.testing.assert_array_equal(f0, 0.0)


def test_bounce_back_mirror_error_is_third_order_in_the_displacement():
    """Fig. 4 / Eq. 17 at a planar wall, phi = tanh(z / (sqrt(2) eps)) sampled on the grid.
    On the exact profile atanh(phi) is proportional to the distance and the reflected
    point is the exact mirror, z_bb = -z_new.  Trilinear interpolation makes phi linear
    inside the wall's grid cells, where atanh(c z) = c z (1 + (c z)^2 / 3 + ...): the two
    distances of the crossing fraction carry relative errors of second order in their
    size, so the mirror is off by a term of third order in the step's displacement,
    the same on every grid.  Halving the start height and the velocity divides the
    error by 8."""
    for h in (0.05, 0.25):
        w = inputs.channel(3.0, 3.0, 3.0, seed=0, h=h)
        f = _field(w)
        p = oracle.Params(box=w.box, a_ff=0.0, gamma=0.0, sigma=0.0, dt=0.01)
        errs = []
        for k in (1.0, 0.5, 0.25, 0.125):
            r0 = np.array([1.13, 1.31, 0.0137 * k])
            v0 = np.array([0.7, -1.1, -3.3 * k])
            s1, refl = oracle.step(oracle.init_forces(_lone_particle(w, r0, v0), p), p, f,
                                   return_reflected=True)
            assert refl[0]
            z_new = r0[2] + v0[2] * p.dt
            errs.append(abs(s1.pos[0, 2] + z_new))
        ratios = np.array(errs[:-1]) / np.array(errs[1:])
        assert np.all((ratios > 7.5) & (ratios < 8.5)), (h, errs)
        assert errs[0] < 1e-5  # displacement 0.033 r_c: the mirror is right to 3e-4 of it
