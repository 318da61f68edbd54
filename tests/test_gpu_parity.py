"""Parity of the CUDA library (through its C ABI) with the FP64 oracle.

Each comparison starts GPU and oracle from the same binary32 state, read back from
the GPU, and compares one step (drift, reflection, cell list, forces, closing
kick) particle by particle under the tolerances of tests/parity_helpers.py.
Sizes run from a 3x3x3 box (the smallest cell grid, every cell on the periodic
seam) through several thread blocks with a ragged tail up to the benchmark's
channel of about one million fluid particles.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1807_09896_gb300 import dpd, inputs
from parity_helpers import (check_forces, compare_one_step, first_newton3_variant, force_scales,
                            gpu_state,
                            make_system, params_for)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1807_09896_gb300 import _build
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()


def _field(w):
    return oracle.Field(w.phi, w.h)


def _initial_force_parity(w, p, newton3=False):
    s = make_system(w, p, load=False)
    _use_algorithm(s, newton3)
    s.set_particles(w.pos4(), w.vel4(), w.id, w.type)
    pos, vel, frc, types = gpu_state(s)
    ids = np.arange(len(pos))
    vt = vel.astype(np.float64)
    vt[types != 0] = 0.0
    f_or, fabs = force_scales(pos.astype(np.float64), vt, ids, types, p, 0)
    err = check_forces(frc, f_or, fabs, types, what="f(0)")
    # the GPU keeps the input state exactly
    np.testing.assert_array_equal(pos, w.pos)
    np.testing.assert_array_equal(vel[types == 0], w.vel[w.type == 0])
    return s, err


CASES = {
    "channel_c1": lambda: inputs.channel(10.0, 10.0, 10.0, seed=0),
    "channel_ragged": lambda: inputs.channel(7.0, 5.0, 5.0, seed=3),
    "bulk_3cube": lambda: inputs.bulk(3.0, seed=1),
    "bulk_no_walls": lambda: inputs.bulk((4.0, 5.0, 6.0), seed=2),
    "channel_tiles": lambda: inputs.channel(24.0, 16.0, 12.0, seed=4),
    "sphere_pack": lambda: inputs.sphere_pack(12.0, 3, 2.0, 3.0, seed=5),
}


@pytest.mark.parametrize("newton3", [False, True])
@pytest.mark.parametrize("name", sorted(CASES))
def test_initial_force_matches_oracle(name, newton3):
    w = CASES[name]()
    p = params_for(w, g=(0.02, 0.0, 0.0), seed=123)
    s, err = _initial_force_parity(w, p, newton3)
    assert err < 1e-5
    s.close()


def _use_algorithm(s, newton3):
    s.set_option("force_variant", first_newton3_variant(s) if newton3 else 0)
    assert bool(s.get_option("force_newton3")) == newton3


@pytest.mark.parametrize("newton3", [False, True])
@pytest.mark.parametrize("name", sorted(CASES))
def test_steps_match_oracle_from_identical_state(name, newton3):
    w = CASES[name]()
    p = params_for(w, g=(0.02, 0.0, 0.0), seed=7)
    s = make_system(w, p)
    _use_algorithm(s, newton3)
    field = _field(w)
    seen_reflections = 0
    for block in range(4):
        r = compare_one_step(s, w, p, field, label=f"{name} step {block}")
        seen_reflections += r["reflections"]
        s.step(4)  # let the GPU run on, then compare again from its own state
    if "channel" in name:
        assert seen_reflections > 0 or w.n < 2000
    s.close()


def test_reflect_variant_literal_eq17():
    w = inputs.channel(6.0, 5.0, 4.0, seed=8)
    p = params_for(w, g=(0.05, 0.0, 0.0), seed=3, reflect_variant=1)
    s = make_system(w, p)
    for _ in range(3):
        compare_one_step(s, w, p, _field(w), label="variant 1")
        s.step(5)
    s.close()


def test_body_force_and_parameters_enter_like_the_oracle():
    w = inputs.channel(6.0, 6.0, 5.0, seed=9)
    p = params_for(w, g=(0.3, -0.1, 0.05), seed=11, a_ff=18.75, a_fs=40.0, gamma=2.0,
                   sigma=1.5, lam=0.5, dt=0.005)
    s = make_system(w, p)
    for _ in range(3):
        compare_one_step(s, w, p, _field(w), label="params")
        s.step(3)
    s.close()


def test_edge_positions_on_the_box_faces():
    w = inputs.channel(5.0, 4.0, 4.0, seed=10)
    pos = w.pos.copy()
    fluid = np.nonzero(w.type == 0)[0]
    L = np.asarray(w.box, np.float32)
    pos[fluid[0], 0] = 0.0
    pos[fluid[1], 0] = np.nextafter(L[0], np.float32(0))
    pos[fluid[2], 1] = 0.0
    pos[fluid[3], 1] = np.nextafter(L[1], np.float32(0))
    w.pos = pos
    p = params_for(w, seed=5)
    s, err = _initial_force_parity(w, p)
    compare_one_step(s, w, p, _field(w), label="faces")
    s.close()


def test_empty_and_all_solid_systems():
    w = inputs.channel(4.0, 4.0, 3.0, seed=1)
    p = params_for(w)
    s = make_system(w, p, load=False)
    s.set_particles(np.zeros((0, 4), np.float32), np.zeros((0, 4), np.float32),
                    np.zeros(0, np.int32), np.zeros(0, np.uint8))
    s.step(3)
    st = s.stats()
    assert st[4] == 0 and st[7] == 3
    solid = w.type != 0
    ns = int(solid.sum())
    s.set_particles(w.pos4()[solid], w.vel4()[solid], np.arange(ns, dtype=np.int32),
                    np.ones(ns, np.uint8))
    s.step(2)
    pos, vel, frc, types = gpu_state(s)
    np.testing.assert_array_equal(pos, w.pos[solid])
    assert np.all(vel == 0) and np.all(frc == 0)
    s.close()


def test_deterministic_and_graph_replay_is_bitwise_equal():
    w = inputs.channel(12.0, 8.0, 6.0, seed=12)
    p = params_for(w, g=(0.02, 0, 0), seed=1)
    a = make_system(w, p, use_graph=1, graph_steps=10)
    b = make_system(w, p, use_graph=0)
    c = make_system(w, p, use_graph=1, graph_steps=4)
    for s in (a, b, c):
        s.step(37)
    ra, rb, rc = (gpu_state(s) for s in (a, b, c))
    for x, y, z in zip(ra, rb, rc):
        np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(x, z)
    for s in (a, b, c):
        s.close()


def test_input_order_does_not_change_the_trajectory():
    """Particles are stored by id when loaded and every cell keeps them in a fixed
    order from then on, so a shuffled input steps to the same bits."""
    w = inputs.channel(10.0, 8.0, 6.0, seed=21)
    p = params_for(w, g=(0.02, 0, 0), seed=3)
    a = make_system(w, p, load=False)
    b = make_system(w, p, load=False)
    a.set_particles(w.pos4(), w.vel4(), w.id, w.type)
    perm = np.random.default_rng(5).permutation(len(w.id))
    b.set_particles(w.pos4()[perm], w.vel4()[perm], w.id[perm], w.type[perm])
    for s in (a, b):
        s.step(9)
    for x, y in zip(gpu_state(a), gpu_state(b)):
        np.testing.assert_array_equal(x, y)
    for s in (a, b):
        s.close()


def test_momentum_conserved_in_periodic_fluid():
    w = inputs.bulk(8.0, seed=4)
    p = params_for(w, seed=2)
    s = make_system(w, p)
    pos, vel, frc, types = gpu_state(s)
    fsum = np.abs(frc.astype(np.float64).sum(0))
    assert fsum.max() <= len(pos) * np.finfo(np.float32).eps * np.abs(frc).max()
    p0 = s.stats()[:3].copy()
    s.step(50)
    p1 = s.stats()[:3]
    # each step adds at most N * eps32 * max|dt F| of round-off momentum
    assert np.abs(p1 - p0).max() < 50 * len(pos) * 1e-6


def test_profile_sums_match_oracle():
    w = inputs.channel(8.0, 6.0, 6.0, seed=13)
    p = params_for(w, g=(0.05, 0, 0), seed=3)
    s = make_system(w, p)
    s.step(10)
    pos, vel, frc, types = gpu_state(s)
    nb, lo, hi = 24, 0.0, 6.0
    gpu = s.profile(2, nb, lo, hi, mode=1)
    ref = oracle.profile(pos, vel.astype(np.float64), types, 2, nb, lo, hi)
    np.testing.assert_array_equal(gpu[:, 0], ref[:, 0])  # counts: exact
    np.testing.assert_allclose(gpu[:, 1:], ref[:, 1:], rtol=1e-12, atol=1e-9)
    # accumulation: a second sample of the same state doubles every sum
    gpu2 = s.profile(2, nb, lo, hi, mode=0)
    np.testing.assert_allclose(gpu2, 2 * gpu, rtol=1e-12, atol=1e-9)
    # automatic sampling inside dpd_step
    s.profile(2, nb, lo, hi, mode=3)
    s.set_option("sample_every", 2)
    s.step(6)
    acc = s.profile(2, nb, lo, hi, mode=2)
    assert acc[:, 0].sum() == 3 * (types == 0).sum()
    s.close()


def test_error_codes_are_returned_not_faults():
    w = inputs.channel(5.0, 5.0, 4.0, seed=14)
    p = params_for(w)
    s = make_system(w, p, load=False)
    with pytest.raises(dpd.DPDError) as e:
        s.step(1)
    assert e.value.code == dpd.DPD_ESTATE
    bad_ids = w.id.copy()
    bad_ids[1] = bad_ids[0]
    with pytest.raises(dpd.DPDError) as e:
        s.set_particles(w.pos4(), w.vel4(), bad_ids, w.type)
    assert e.value.code == dpd.DPD_EINVAL
    pos = w.pos4()
    fl = np.nonzero(w.type == 0)[0][0]
    pos[fl, 2] = w.gap + 1.0  # a fluid particle in the middle of the solid
    with pytest.raises(dpd.DPDError) as e:
        s.set_particles(pos, w.vel4(), w.id, w.type)
    assert e.value.code == dpd.DPD_ELOST
    s.set_particles(w.pos4(), w.vel4(), w.id, w.type)
    s.set_option("band_margin", 0.001)  # drifts of ~0.01 exceed it
    with pytest.raises(dpd.DPDError) as e:
        s.step(2)
    assert e.value.code == dpd.DPD_EBAND
    with pytest.raises(dpd.DPDError) as e:
        s.set_option("no_such_option", 1.0)
    assert e.value.code == dpd.DPD_EINVAL
    s.close()


def test_no_fluid_particle_enters_the_solid_over_a_run():
    w = inputs.channel(10.0, 10.0, 10.0, seed=15)
    p = params_for(w, g=(0.02, 0, 0), seed=4)
    s = make_system(w, p)
    field = _field(w)
    for _ in range(10):
        s.step(50)
        pos, vel, frc, types = gpu_state(s)
        assert oracle.phi_many(field, pos[types == 0]).min() >= 0.0
    assert s.stats()[5] > 0
    s.close()


@pytest.mark.parametrize("newton3", [False, True])
def test_full_size_channel_one_million(newton3):
    """The benchmark's workload (channel 80 x 64 x 64 gap, ~983k fluid particles)
    in the benchmark's launch configuration (graph replay): after 20 graph steps
    one more step is compared particle by particle with the oracle."""
    w = inputs.channel(80.0, 64.0, 64.0, seed=0)
    p = params_for(w, g=(0.01, 0.0, 0.0), seed=0)
    s, err = _initial_force_parity(w, p, newton3)
    s.set_option("use_graph", 1)
    s.set_option("graph_steps", 20)
    s.step(20)
    r = compare_one_step(s, w, p, _field(w), label="1M")
    assert r["reflections"] > 0
    s.close()


def test_every_force_launch_shape_gives_bitwise_identical_steps():
    """Within each force algorithm every launch shape gives the same bits; the two
    algorithms (full shell in binary32, Newton's third law in fixed point) agree to
    rounding."""
    w = inputs.channel(9.0, 7.0, 6.0, seed=16)
    p = params_for(w, g=(0.02, 0, 0), seed=6)
    ref, f0 = {}, {}
    nv = int(make_system(w, p, load=False).get_option("force_variants"))
    for v in range(nv):
        s = make_system(w, p, load=False, force_variant=v)
        fam = bool(s.get_option("force_newton3"))
        s.set_particles(w.pos4(), w.vel4(), w.id, w.type)
        f0.setdefault(fam, gpu_state(s)[2])
        s.step(7)
        st = gpu_state(s)
        if fam not in ref:
            ref[fam] = st
        else:
            for x, y in zip(ref[fam], st):
                np.testing.assert_array_equal(x, y)
        s.close()
    assert set(ref) == {False, True}
    # from the same state the two algorithms' forces differ by the rounding of the sums
    assert np.abs(f0[False] - f0[True]).max() < 1e-4


def test_autotune_keeps_results_and_picks_a_shape():
    """Tuning leaves the state and counters as they were; afterwards the system
    steps like any system using the chosen shape."""
    w = inputs.channel(10.0, 8.0, 6.0, seed=17)
    p = params_for(w, seed=8)
    a = make_system(w, p)
    b = make_system(w, p)
    before = gpu_state(a), a.stats()
    chosen, ms = dpd.dpd_autotune(a.h, 2)
    assert 0 <= chosen < len(ms) and all(m > 0 for m in ms)
    assert a.get_option("force_variant") == chosen
    for x, y in zip(before[0], gpu_state(a)):
        np.testing.assert_array_equal(x, y)
    after = a.stats()
    np.testing.assert_array_equal(before[1][5:], after[5:])  # reflections, fallbacks, step
    np.testing.assert_allclose(before[1][:5], after[:5], rtol=1e-12)  # FP64 atomic sums
    b.set_option("force_variant", chosen)
    a.step(9)
    b.step(9)
    for x, y in zip(gpu_state(a), gpu_state(b)):
        np.testing.assert_array_equal(x, y)


def test_moving_walls_match_the_oracle():
    """Walls moving at v_wall (Sec. II.C: reflection gives 2 v_wall - v, and frozen
    particles enter the dissipative force with v_wall)."""
    w = inputs.channel(6.0, 5.0, 5.0, seed=18)
    p = params_for(w, seed=12, v_wall=(0.4, -0.2, 0.0))
    s = make_system(w, p, v_wall_x=0.4, v_wall_y=-0.2)
    for _ in range(3):
        compare_one_step(s, w, p, _field(w), label="moving walls")
        s.step(5)
    s.close()


def test_couette_walls_match_the_oracle():
    """Walls sliding at different velocities (wall velocity field v_wall + d S along
    z, reading R18): reflection with the crossed wall's velocity, frozen particles
    moving with theirs and entering the dissipative force with it."""
    w = inputs.channel(6.0, 5.0, 5.0, seed=21)
    p = params_for(w, seed=14, v_wall=(0.1, 0.0, 0.0), shear=(0.3, -0.12, 0.0), shear_axis=2,
                   shear_ref=2.5)
    s = make_system(w, p)
    for _ in range(3):
        compare_one_step(s, w, p, _field(w), label="couette walls")
        s.step(5)
    s.close()


def test_shear_along_its_own_axis_is_rejected():
    w = inputs.channel(6.0, 5.0, 5.0, seed=21)
    s = make_system(w, params_for(w), load=False)
    with pytest.raises(dpd.DPDError):
        s.set_option("shear_z", 0.1)  # default axis z: would move the walls through phi
    s.set_option("shear_x", 0.1)
    with pytest.raises(dpd.DPDError):
        s.set_option("shear_axis", 0)
    s.close()


@pytest.mark.parametrize("dim", [3, 2])
def test_attractive_repulsive_force_law_matches_the_oracle(dim):
    """The pair energy of Eq. 22 with the spline of Eq. 23 (force -dE/dr, Eq. 24) and
    the paper's wetting parameters (kBT 0.5, gamma 4.5, fluid-solid strengths twice
    the fluid-fluid ones), in a channel: fluid-fluid and fluid-solid pairs, seams."""
    w = inputs.channel(6.0, 5.0, 5.0, seed=22, kBT=0.5)
    p = params_for(w, seed=15, force_law=1, sph_dim=dim, kBT=0.5, gamma=4.5,
                   sigma=math.sqrt(2 * 4.5 * 0.5), g=(0.02, 0.0, 0.0))
    s = make_system(w, p)
    for _ in range(3):
        compare_one_step(s, w, p, _field(w), label=f"force law 1, D={dim}")
        s.step(5)
    s.close()


def test_batch_rejects_mixed_force_laws():
    w = inputs.channel(6.0, 5.0, 5.0, seed=22)
    a = make_system(w, params_for(w))
    b = make_system(w, params_for(w, force_law=1))
    with pytest.raises(dpd.DPDError):
        dpd.Batch([a, b])
    a.close()
    b.close()


def test_newton3_steps_repeat_bitwise():
    """The Newton's-third-law shapes scatter -f_ij with atomics whose arrival order varies
    from run to run; the fixed-point sums do not depend on it (and each particle's own
    binary32 sum runs in the fixed cell order), so two runs agree bit for bit."""
    w = inputs.channel(12.0, 9.0, 8.0, seed=24)
    p = params_for(w, g=(0.02, 0.0, 0.0), seed=13)
    runs = []
    for _ in range(2):
        s = make_system(w, p)
        _use_algorithm(s, True)
        s.set_option("use_graph", 0)
        s.step(25)
        runs.append((gpu_state(s), s.stats()[5:]))
        s.close()
    for x, y in zip(runs[0][0], runs[1][0]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(runs[0][1], runs[1][1])


def test_a_cell_beyond_48_particles_returns_overflow_not_a_fault():
    """The per-cell sort holds at most 48 particles per cell (eight times more than
    rho = 3 ever puts there); a crowded cell is reported as DPD_EOVERFLOW."""
    w = inputs.bulk(5.0, seed=3)
    pos = w.pos4()
    rng = np.random.default_rng(0)
    pos[:60, :3] = 2.0 + rng.uniform(0.0, 1.0, size=(60, 3))  # 60 particles in one unit cell
    s = make_system(w, params_for(w), load=False)
    with pytest.raises(dpd.DPDError) as e:
        s.set_particles(pos, w.vel4(), w.id, w.type)
        s.step(1)
    assert e.value.code == dpd.DPD_EOVERFLOW
    s.set_particles(w.pos4(), w.vel4(), w.id, w.type)  # a valid state clears it
    s.step(2)
    s.close()
