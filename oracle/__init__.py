"""FP64 CPU oracle for the phase-field no-slip DPD time step (arXiv:1807.09896).

TEST INFRASTRUCTURE ONLY.  This package exists so that the tests, the smoke
check and the benchmark's CPU-baseline leg can check the CUDA library against a
plain, slow, obviously correct restatement of the paper.  Nothing in the product
path imports it, and it imports nothing from the product package.

The arithmetic lives in ``dpd_oracle.c`` (built by ``oracle/build.py``); this
module only marshals numpy arrays into it.  Citations:

* pair noise ``xi_ij`` (Eq. 7): Philox4x32-10 + Box-Muller, ``philox``/``xi``;
* pair force (Eqs. 3-10): ``forces``;
* time step (Sec. II.A integrator, ref. 35) with bounce-back reflection
  (Sec. II.C, Eq. 17, Fig. 4): ``step``;
* particle phase field by trilinear interpolation (Sec. II.C): ``phi_at``;
* velocity-profile sums (Sec. III.A): ``profile``.

Parity status of each function is recorded at the top of ``dpd_oracle.c`` and in
the tests under ``tests/test_oracle_*.py``.  The absolute viscosity of the 3-D
fluid is "parity unpinned": the paper prints only 2-D values.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_P_NAMES = [
    "Lx", "Ly", "Lz", "a_ff", "a_fs", "a_sf", "a_ss", "gamma", "sigma", "kBT", "dt",
    "lam", "gx", "gy", "gz", "vwx", "vwy", "vwz", "reflect_variant",
    "shx", "shy", "shz", "sh_axis", "sh_ref",
    "force_law", "S_r_ff", "S_a_ff", "S_r_fs", "S_a_fs", "r0_r", "r0_a", "sph_dim",
]

_lib = None


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_philox4x32_10.restype = None
        L.or_u01.argtypes = [ctypes.c_uint32]
        L.or_u01.restype = ctypes.c_double
        L.or_xi.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                            ctypes.c_uint64]
        L.or_xi.restype = ctypes.c_double
        L.or_phi_at.argtypes = [f32p, i32p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double]
        L.or_phi_at.restype = ctypes.c_double
        L.or_pairs.argtypes = [ctypes.c_int, f64p, f64p, ctypes.c_int, ctypes.c_long, i32p]
        L.or_pairs.restype = ctypes.c_long
        L.or_forces.argtypes = [ctypes.c_int, f64p, f64p, i32p, u8p, f64p, ctypes.c_uint32,
                                ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, f64p]
        L.or_forces.restype = ctypes.c_int
        L.or_forces_sel.argtypes = [ctypes.c_int, f64p, f64p, i32p, u8p, f64p, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                    i32p, f64p, f64p]
        L.or_forces_sel.restype = ctypes.c_int
        L.or_phi_many.argtypes = [f32p, i32p, ctypes.c_double, ctypes.c_long, f64p, f64p]
        L.or_phi_many.restype = None
        L.or_step.argtypes = [ctypes.c_int, f64p, f64p, f64p, i32p, u8p, f64p, f32p, i32p,
                              ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                              ctypes.c_int, u8p, i64p, f64p]
        L.or_step.restype = ctypes.c_int
        L.or_wall_velocities.argtypes = [ctypes.c_int, f64p, u8p, f64p, f64p]
        L.or_wall_velocities.restype = None
        for fn in ("or_sph_W", "or_sph_dWdr"):
            getattr(L, fn).argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
            getattr(L, fn).restype = ctypes.c_double
        L.or_sph_energy.argtypes = [f64p, ctypes.c_double, ctypes.c_int]
        L.or_sph_energy.restype = ctypes.c_double
        L.or_init_particles.argtypes = [ctypes.c_long, f64p, ctypes.c_double, ctypes.c_uint64,
                                        ctypes.c_uint32, ctypes.c_double, ctypes.c_int, f32p, i32p,
                                        ctypes.c_double, f64p, u8p, f64p, f64p, u8p, i64p]
        L.or_init_particles.restype = ctypes.c_long
        L.or_profile.argtypes = [ctypes.c_int, f32p, f64p, u8p, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_double, f64p]
        L.or_profile.restype = None
        L.or_num_threads.argtypes = []
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


@dataclass
class Params:
    """Physical and numerical parameters of one DPD system (DPD units, r_c = m = 1)."""

    box: tuple = (10.0, 10.0, 12.0)
    a_ff: float = 25.0
    a_fs: float = 25.0
    gamma: float = 4.5
    sigma: float = 3.0
    kBT: float = 1.0
    dt: float = 0.01
    lam: float = 0.65
    g: tuple = (0.0, 0.0, 0.0)
    v_wall: tuple = (0.0, 0.0, 0.0)
    reflect_variant: int = 0
    seed: int = 0
    sys: int = 0
    shear: tuple = (0.0, 0.0, 0.0)  # d v_wall / d r_axis (plane Couette walls)
    shear_axis: int = 2
    shear_ref: float = 0.0
    # attractive/repulsive SPH-kernel force (Eqs. 22-24), the paper's wetting values
    force_law: int = 0
    S_r_ff: float = 37.5
    S_a_ff: float = 18.75
    S_r_fs: float = 75.0
    S_a_fs: float = 37.5
    r0_r: float = 0.73
    r0_a: float = 1.0
    sph_dim: int = 3

    def flat(self) -> np.ndarray:
        v = [*self.box, self.a_ff, self.a_fs, self.a_fs, 0.0, self.gamma, self.sigma, self.kBT,
             self.dt, self.lam, *self.g, *self.v_wall, float(self.reflect_variant),
             *self.shear, float(self.shear_axis), self.shear_ref,
             float(self.force_law), self.S_r_ff, self.S_a_ff, self.S_r_fs, self.S_a_fs,
             self.r0_r, self.r0_a, float(self.sph_dim)]
        assert len(v) == len(_P_NAMES)
        return np.asarray(v, dtype=np.float64)


@dataclass
class Field:
    """Phase field on a periodic grid: node (i, j, k) sits at (i, j, k) * h."""

    grid: np.ndarray  # float32, shape (nz, ny, nx), x fastest
    h: float

    @property
    def dims(self) -> np.ndarray:
        nz, ny, nx = self.grid.shape
        return np.asarray([nx, ny, nz], dtype=np.int32)


@dataclass
class State:
    """Particle state in id order: r, v, pair force f (without the body force)."""

    pos: np.ndarray
    vel: np.ndarray
    frc: np.ndarray
    id: np.ndarray
    type: np.ndarray
    step: int = 0
    stats: dict = field(default_factory=lambda: {"reflections": 0, "fallbacks": 0})

    def copy(self) -> "State":
        return State(self.pos.copy(), self.vel.copy(), self.frc.copy(), self.id.copy(),
                     self.type.copy(), self.step, dict(self.stats))


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 128-bit counter under one 64-bit key."""
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_c(ctr, np.uint32), _c(key, np.uint32), out)
    return out


def u01(x: int) -> float:
    return lib().or_u01(int(x) & 0xFFFFFFFF)


def xi(id_a: int, id_b: int, step: int, sys: int, seed: int) -> float:
    """Gaussian pair noise of Eq. 7 for the pair (id_a, id_b) at `step`."""
    return lib().or_xi(id_a, id_b, step, sys, seed)


def phi_at(f: Field, pts) -> np.ndarray:
    """Trilinear periodic interpolation of the phase field at points (n, 3)."""
    pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    g = _c(f.grid, np.float32).reshape(-1)
    d = f.dims
    L = lib()
    return np.array([L.or_phi_at(g, d, f.h, p[0], p[1], p[2]) for p in pts])


def pairs(pos, box, method: int = 0) -> np.ndarray:
    """All unordered pairs (i < j) closer than r_c = 1, lexicographic rows."""
    pos = _c(pos, np.float64)
    n = len(pos)
    L = _c(box, np.float64)
    cap = max(16, n * 64)
    out = np.zeros(2 * cap, np.int32)
    m = lib().or_pairs(n, pos.reshape(-1), L, method, cap, out)
    if m < 0:
        raise ValueError("box too small for the cell list (each edge must be >= 3 r_c)")
    if m > cap:
        raise RuntimeError("pair buffer too small")
    return out[: 2 * m].reshape(m, 2)


def forces(pos, vt, ids, types, p: Params, step: int, method: int = 1) -> np.ndarray:
    """Total pair force on every particle (Eq. 2) at predicted velocities vt."""
    pos = _c(pos, np.float64)
    n = len(pos)
    f = np.zeros((n, 3), np.float64)
    rc = lib().or_forces(n, pos.reshape(-1), _c(vt, np.float64).reshape(-1), _c(ids, np.int32),
                         _c(types, np.uint8), p.flat(), step, p.sys, p.seed, method,
                         f.reshape(-1))
    if rc != 0:
        raise RuntimeError(f"or_forces failed ({rc})")
    return f


def forces_sel(pos, vt, ids, types, p: Params, step: int, sel, method: int = 1):
    """Pair force (Eq. 2) on the particles listed in `sel` only, and for each of
    them sum_j |f_ij| (the scale a force error is measured against)."""
    pos = _c(pos, np.float64)
    sel = _c(sel, np.int32)
    f = np.zeros((len(sel), 3), np.float64)
    fabs = np.zeros(len(sel), np.float64)
    rc = lib().or_forces_sel(len(pos), pos.reshape(-1), _c(vt, np.float64).reshape(-1),
                             _c(ids, np.int32), _c(types, np.uint8), p.flat(), step, p.sys, p.seed,
                             method, len(sel), sel, f.reshape(-1), fabs)
    if rc != 0:
        raise RuntimeError(f"or_forces_sel failed ({rc})")
    return f, fabs


def phi_many(f: Field, pts) -> np.ndarray:
    """Phase field at many points (n, 3), computed in C."""
    pts = _c(np.atleast_2d(pts), np.float64)
    out = np.zeros(len(pts), np.float64)
    lib().or_phi_many(_c(f.grid, np.float32).reshape(-1), f.dims, f.h, len(pts), pts.reshape(-1), out)
    return out


def init_forces(s: State, p: Params, method: int = 1) -> State:
    """f(0): the pair force at the initial state, with the predicted velocity equal to v(0)."""
    s = s.copy()
    vt = s.vel.copy()
    solid = s.type != 0
    vt[solid] = wall_velocities(s.pos, s.type, p)[solid]
    s.frc = forces(s.pos, vt, s.id, s.type, p, s.step, method)
    return s


def sph_W(r: float, r0: float, D: int) -> float:
    """Smoothing function of Eq. 23 with support scale r0 in D dimensions."""
    return lib().or_sph_W(float(r), float(r0), int(D))


def sph_dWdr(r: float, r0: float, D: int) -> float:
    """dW/dr of Eq. 23."""
    return lib().or_sph_dWdr(float(r), float(r0), int(D))


def sph_energy(p: Params, r: float, fluid_solid: bool = False) -> float:
    """Pair energy of Eq. 22 with the strengths of p."""
    return lib().or_sph_energy(p.flat(), float(r), int(bool(fluid_solid)))


def init_particles(box, rho: float, kBT: float, seed: int, phi_min: float, field=None, sys: int = 0):
    """Particle set-up from the phase field (Sec. II.C): round(rho V) random sites,
    classified by phi (fluid >= 0 > solid > phi_min >= removed), mean fluid velocity
    removed.  Returns a dict: pos, vel, type, site (kept particles in site order) and
    site_phi, site_type (every site)."""
    L = np.asarray(box, np.float64)
    n0 = int(np.floor(rho * L.prod() + 0.5))
    m = max(n0, 1)
    site_phi = np.zeros(m); site_type = np.zeros(m, np.uint8)
    pos = np.zeros((m, 3)); vel = np.zeros((m, 3)); typ = np.zeros(m, np.uint8)
    site = np.zeros(m, np.int64)
    if field is None:
        grid, dims, h, have = np.ones(1, np.float32), np.ones(3, np.int32), 1.0, 0
    else:
        grid, dims, h, have = _c(field.grid, np.float32).reshape(-1), field.dims, field.h, 1
    n = lib().or_init_particles(n0, _c(L, np.float64), float(kBT), int(seed), int(sys), float(phi_min),
                                have, grid, dims, float(h), site_phi, site_type, pos.reshape(-1),
                                vel.reshape(-1), typ, site)
    return {"pos": pos[:n], "vel": vel[:n], "type": typ[:n], "site": site[:n],
            "site_phi": site_phi[:n0], "site_type": site_type[:n0], "n0": n0}


def wall_velocities(pos, types, p: Params) -> np.ndarray:
    """Wall velocity v_w(r) of every solid particle (zero rows for fluid), reading R18."""
    pos = _c(np.atleast_2d(pos), np.float64)
    out = np.zeros((len(pos), 3), np.float64)
    lib().or_wall_velocities(len(pos), pos.reshape(-1), _c(types, np.uint8), p.flat(), out.reshape(-1))
    return out


def step(s: State, p: Params, f: Field, method: int = 1, return_reflected: bool = False,
         return_wall_velocity: bool = False):
    """Advance the state by one time step; the new force uses counter step+1.

    return_reflected adds the per-particle reflection flags; return_wall_velocity
    adds the wall velocity each particle met this step (solid particles: their own;
    reflected particles: at the crossing point; others: zero)."""
    s = s.copy()
    n = len(s.pos)
    refl = np.zeros(n, np.uint8)
    stats = np.zeros(2, np.int64)
    vwall = np.zeros((n, 3), np.float64)
    pos = _c(s.pos, np.float64)
    vel = _c(s.vel, np.float64)
    frc = _c(s.frc, np.float64)
    rc = lib().or_step(n, pos.reshape(-1), vel.reshape(-1), frc.reshape(-1), _c(s.id, np.int32),
                       _c(s.type, np.uint8), p.flat(), _c(f.grid, np.float32).reshape(-1),
                       f.dims, f.h, s.step + 1, p.sys, p.seed, method, refl, stats,
                       vwall.reshape(-1))
    if rc != 0:
        raise RuntimeError(f"or_step failed ({rc})")
    s.pos, s.vel, s.frc = pos, vel, frc
    s.step += 1
    s.stats = {"reflections": s.stats["reflections"] + int(stats[0]),
               "fallbacks": s.stats["fallbacks"] + int(stats[1])}
    out = (s,)
    if return_reflected:
        out += (refl.astype(bool),)
    if return_wall_velocity:
        out += (vwall,)
    return out if len(out) > 1 else s


def profile(pos_f32, vel, types, axis: int, nbins: int, lo: float, hi: float,
            out: np.ndarray | None = None) -> np.ndarray:
    """Per-bin {count, sum vx, sum vy, sum vz, sum |v|^2} over fluid particles.

    ``pos_f32`` are binary32 positions (the bin decision is taken in binary32).
    """
    if out is None:
        out = np.zeros((nbins, 5), np.float64)
    pos4 = np.zeros((len(pos_f32), 4), np.float32)
    pos4[:, :3] = np.asarray(pos_f32, dtype=np.float32)[:, :3]
    lib().or_profile(len(pos4), pos4.reshape(-1), _c(vel, np.float64).reshape(-1),
                     _c(types, np.uint8), axis, nbins, lo, hi, out.reshape(-1))
    return out


def num_threads() -> int:
    return lib().or_num_threads()
