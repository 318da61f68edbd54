"""Helpers for comparing the CUDA library with the FP64 oracle on identical state.

Tolerances (binary32 arithmetic on the GPU against binary64 in the oracle):

* pair force: |f_gpu - f_or| <= 1e-5 * sum_j |f_ij| + 1e-6, per particle and
  component, with the oracle evaluated at the GPU's binary32 positions.  sum_j
  |f_ij| is the scale of the terms being added, so the bound is a relative error
  of the sum's terms, meaningful even where f ~ 0.
* position: |r_gpu - r_or| (minimum image) <= 1e-5 |dr| + 2 ulp32(L_max): the
  GPU adds a binary32 drift to a binary32 position.
* velocity: |v_gpu - v_or| <= 1e-5 (|v| + dt/2 (S(t) + S(t+dt))) + 4 ulp32(|v|),
  with S the force scales above.
* reflection decisions agree except where |phi(r')| < 1e-5 (the sign of phi is
  then decided by rounding); such particles and their neighbours within r_c
  are left out of the force and velocity comparison.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_1807_09896_gb300 import dpd

F_REL = 1e-5
F_ABS = 1e-6
PHI_AMBIGUOUS = 1e-5


def params_for(w, g=(0.0, 0.0, 0.0), seed=0, **kw):
    return oracle.Params(box=w.box, g=g, seed=seed, **kw)


def make_system(w, p: oracle.Params, load=True, **options):
    s = dpd.System(w.box, a_ff=p.a_ff, a_fs=p.a_fs, gamma=p.gamma, sigma=p.sigma, kBT=p.kBT,
                   dt=p.dt, g=p.g)
    s.set_option("lambda", p.lam)
    s.set_option("seed", p.seed)
    s.set_option("system", p.sys)
    s.set_option("reflect_variant", p.reflect_variant)
    for c, v in zip("xyz", p.v_wall):
        s.set_option(f"v_wall_{c}", v)
    s.set_option("shear_axis", p.shear_axis)
    s.set_option("shear_ref", p.shear_ref)
    for c, v in zip("xyz", p.shear):
        s.set_option(f"shear_{c}", v)
    for k in ("force_law", "S_r_ff", "S_a_ff", "S_r_fs", "S_a_fs", "r0_r", "r0_a", "sph_dim"):
        s.set_option(k, getattr(p, k))
    for k, v in options.items():
        s.set_option(k, v)
    dpd.dpd_set_phase_field(s.h, w.phi, w.h)
    if load:
        s.set_particles(w.pos4(), w.vel4(), w.id, w.type)
    return s


def first_newton3_variant(s) -> int:
    """Index of the first force launch shape that evaluates each pair once."""
    keep = int(s.get_option("force_variant"))
    try:
        for v in range(int(s.get_option("force_variants"))):
            s.set_option("force_variant", v)
            if s.get_option("force_newton3"):
                return v
    finally:
        s.set_option("force_variant", keep)
    raise AssertionError("no Newton's-third-law force shape")


def gpu_state(s):
    pos4, vel4, f4, ids, types = s.state()
    assert np.array_equal(ids, np.arange(len(ids)))
    return pos4[:, :3].copy(), vel4[:, :3].copy(), f4[:, :3].copy(), types


def oracle_state(pos, vel, frc, ids, types, step):
    return oracle.State(pos.astype(np.float64), vel.astype(np.float64), frc.astype(np.float64),
                        np.asarray(ids, np.int32), np.asarray(types, np.uint8), step)


def ulp32(x):
    x = np.abs(np.asarray(x, np.float32))
    return np.spacing(x).astype(np.float64)


def min_image(d, box):
    L = np.asarray(box, np.float64)
    return d - L * np.round(d / L)


def check_forces(f_gpu, f_or, fabs, types, skip=None, what="force"):
    fluid = types == 0
    if skip is not None:
        fluid = fluid & ~skip
    err = np.abs(f_gpu.astype(np.float64) - f_or)
    tol = F_REL * fabs[:, None] + F_ABS
    bad = (err > tol) & fluid[:, None]
    if bad.any():
        i, a = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: {bad.any(1).sum()} particles out of tolerance; first i={i} "
                             f"axis={a} gpu={f_gpu[i, a]!r} oracle={f_or[i, a]!r} scale={fabs[i]!r}")
    # solid particles carry no force
    assert np.all(f_gpu[types != 0] == 0.0)
    return float((err[fluid] / (fabs[fluid, None] + 1e-30)).max()) if fluid.any() else 0.0


def force_scales(pos, vt, ids, types, p, step):
    sel = np.arange(len(pos), dtype=np.int32)
    return oracle.forces_sel(pos, vt, ids, types, p, step, sel)


def neighbours_of(mask, pos, box):
    """Particles within r_c of any particle in `mask` (mask included)."""
    out = mask.copy()
    idx = np.nonzero(mask)[0]
    L = np.asarray(box)
    for i in idx:
        d = min_image(pos - pos[i], L)
        out |= (d * d).sum(1) < 1.0
    return out


def compare_one_step(s, w, p, field, label=""):
    """Read the GPU state, advance GPU and oracle one step from it, compare.

    Returns a dict of the largest relative errors seen."""
    pos0, vel0, frc0, types = gpu_state(s)
    step0 = int(s.get_option("step"))
    # the state comes back in id order, so the ids are 0..n-1
    st0 = oracle_state(pos0, vel0, frc0, np.arange(len(pos0)), types, step0)
    stats0 = s.stats()
    s.step(1)
    pos1, vel1, frc1, _ = gpu_state(s)
    gpu_refl = s.state()[1][:, 3] == 1.0  # the library's own flag
    stats1 = s.stats()
    or1, refl, vwall = oracle.step(st0, p, field, return_reflected=True, return_wall_velocity=True)
    moving = bool(np.any(p.v_wall) or np.any(p.shear))

    # would-be positions and their phase field, to find ambiguous reflection decisions
    F0 = st0.frc + np.asarray(p.g)
    dr = p.dt * st0.vel + 0.5 * p.dt * p.dt * F0
    fluid = types == 0
    phi_new = np.ones(len(pos0))
    phi_new[fluid] = oracle.phi_many(field, st0.pos[fluid] + dr[fluid])
    assert not np.any(gpu_refl & ~fluid)
    mismatch = fluid & (gpu_refl != refl)
    both = gpu_refl & refl
    if not np.any(p.shear):
        # a reflected particle leaves with exactly 2 v_wall - v(t), computed in binary32
        v_bb = np.float32(2.0) * np.asarray(p.v_wall, np.float32) - vel0.astype(np.float32)
        assert np.all(vel1[both] == v_bb[both]), f"{label}: reflected velocities"
    else:  # the wall velocity at the crossing point, up to binary32 rounding of that point
        v_bb = 2.0 * vwall - vel0
        assert np.all(np.abs(vel1[both] - v_bb[both]) <= 1e-5 * (1 + np.abs(v_bb[both]))), \
            f"{label}: reflected velocities"

    assert np.all(np.abs(phi_new[mismatch]) < PHI_AMBIGUOUS), (
        f"{label}: reflection decisions differ away from phi = 0: "
        f"{np.nonzero(mismatch & (np.abs(phi_new) >= PHI_AMBIGUOUS))[0][:10]}")
    if not mismatch.any():
        assert int(stats1[5] - stats0[5]) == int(refl.sum()), (stats1[5] - stats0[5], refl.sum())
    skip = neighbours_of(mismatch, or1.pos, w.box) if mismatch.any() else None

    # positions
    dpos = min_image(pos1.astype(np.float64) - or1.pos, w.box)
    tolp = 1e-5 * np.linalg.norm(dr, axis=1)[:, None] + 2 * ulp32(max(w.box))
    okp = (np.abs(dpos) <= tolp) | (mismatch[:, None])
    if not okp.all():
        bad = np.nonzero(~okp.all(1))[0]
        k = bad[np.argmax(np.abs(dpos[bad]).max(1))]
        raise AssertionError(
            f"{label}: {len(bad)} positions differ; worst i={k} gpu={pos1[k]!r} oracle={or1.pos[k]!r} "
            f"start={pos0[k]!r} dr={dr[k]!r} reflected={refl[k]} phi_new={phi_new[k]!r} "
            f"tol={tolp[k]!r}")
    if not moving:
        assert np.all(pos1[~fluid] == pos0[~fluid])
    elif (~fluid).any():  # the solid moves with the wall velocity at each frozen particle
        ds = min_image(pos1[~fluid].astype(np.float64) - pos0[~fluid] - p.dt * vwall[~fluid], w.box)
        assert np.abs(ds).max() < 4 * ulp32(max(w.box))

    # forces at t+dt, evaluated at the GPU's own (binary32) new positions: the oracle's
    # new positions are not rounded to binary32, and the force is steep enough in r
    # that this rounding alone would exceed the force tolerance
    vt = st0.vel + p.lam * p.dt * F0
    vt[refl] = -st0.vel[refl] + 2 * vwall[refl]
    vt[~fluid] = vwall[~fluid]
    ids = np.arange(len(pos0))
    f_ref, fabs1 = force_scales(pos1.astype(np.float64), vt, ids, types, p, step0 + 1)
    _, fabs0 = force_scales(st0.pos, st0.vel, ids, types, p, step0)
    ef = check_forces(frc1, f_ref, fabs1, types, skip=skip, what=f"{label} force")
    keep = fluid if skip is None else fluid & ~skip
    # the oracle's own forces agree with these up to the position rounding
    if keep.any():
        assert np.abs(or1.frc - f_ref)[keep].max() < 1e-2 * max(1.0, np.abs(f_ref).max())

    # velocities: closing half-kick with the reference force (reversed if reflected)
    v_ref = st0.vel + 0.5 * p.dt * (F0 + f_ref + np.asarray(p.g))
    v_ref[refl] = -st0.vel[refl] + 2 * vwall[refl]
    v_ref[~fluid] = 0.0
    dv = np.abs(vel1.astype(np.float64) - v_ref)
    tolv = F_REL * (np.abs(v_ref) + 0.5 * p.dt * (fabs0 + fabs1)[:, None]) + 4 * ulp32(v_ref)
    badv = (dv > tolv) & fluid[:, None]
    if skip is not None:
        badv &= ~skip[:, None]
    assert not badv.any(), f"{label}: velocities differ at {np.nonzero(badv.any(1))[0][:10]}"
    # and the oracle's own velocities agree up to the same position rounding
    if keep.any():
        assert np.abs(or1.vel - v_ref)[keep].max() < 1e-3
    return {"force_rel": ef, "reflections": int(refl.sum()), "ambiguous": int(mismatch.sum())}
