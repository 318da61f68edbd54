"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the benchmark.

This module holds no arithmetic of the method itself: it only draws particle
positions and velocities and tabulates the phase field phi(x) on a grid.  The
phase field is an input of the method; every workload here uses the steady
planar profile of Eq. 14, phi = tanh(d / (sqrt(2) eps)) with d the signed
distance to the solid surface (positive in the fluid) and eps = 0.5, sampled on a
grid of spacing 0.25 r_c (Sec. II.B).

Workloads (DPD units, r_c = 1, rho = 3):

* ``channel(Lx, Ly, H)`` -- a plane channel of fluid gap H between walls at
  z = 0 and z = H.  The box is periodic with Lz = H + 2: a 1 r_c solid layer
  sits below z = 0 (wrapped to z in [H + 1, H + 2)) and above z = H, and the two
  layers meet through the periodic wrap, so the fluid sees walls only.
  Fluid particles are uniform in the gap, solid particles uniform in the
  layers (the paper's frozen boundary particles, Sec. II.C).
* ``channel_2d(Lx, W)`` -- the planar (2-D) channel of Sec. III.A, run as a
  single layer of particles: box Lx x (W + 2 layer) x 3 with every particle at
  z = 1.5 and zero z velocity, walls at y = 0 and y = W.  Pair forces lie along
  the separation, which has no z component, so the layer stays exactly planar
  and the system is a 2-D DPD fluid of areal density rho.
* ``cylinder_2d(L, r)`` -- the square array of parallel cylinders of Sec. III.B, as
  a planar layer like ``channel_2d``: one disk of radius r in a periodic L x L cell.
* ``bulk(L)`` -- a periodic box with no solid (phi = 1 everywhere).
* ``sphere_pack(L, nspheres, rmin, rmax)`` -- a periodic cube holding
  non-overlapping solid spheres; fluid in the pore space, a 1 r_c solid shell
  inside each surface.

Velocities are Maxwellian at k_BT with the mean removed; solid particles are at
rest.  Every array is a deterministic function of the seed (numpy PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

EPS = 0.5      # interface parameter of Eq. 14 used by every workload
GRID_H = 0.25  # phase-field grid spacing


@dataclass
class Workload:
    name: str
    box: tuple          # (Lx, Ly, Lz)
    phi: np.ndarray     # float32 (nz, ny, nx), node (i, j, k) at (i, j, k) * h
    h: float
    pos: np.ndarray     # float32 (n, 3)
    vel: np.ndarray     # float32 (n, 3)
    id: np.ndarray      # int32 (n,), a permutation of 0..n-1
    type: np.ndarray    # uint8 (n,), 0 fluid, 1 solid
    gap: float = 0.0    # channel gap H (0 if not a channel)

    @property
    def n(self) -> int:
        return len(self.pos)

    @property
    def n_fluid(self) -> int:
        return int((self.type == 0).sum())

    @property
    def n_solid(self) -> int:
        return int((self.type != 0).sum())

    def pos4(self) -> np.ndarray:
        p = np.zeros((self.n, 4), np.float32)
        p[:, :3] = self.pos
        return p

    def vel4(self) -> np.ndarray:
        v = np.zeros((self.n, 4), np.float32)
        v[:, :3] = self.vel
        return v


def _phi_from_distance(d: np.ndarray) -> np.ndarray:
    return np.tanh(d / (math.sqrt(2.0) * EPS)).astype(np.float32)


def _grid_dims(box, h):
    dims = []
    for L in box:
        n = int(round(L / h))
        if abs(n * h - L) > 1e-9 * max(1.0, L):
            raise ValueError(f"box edge {L} is not a whole number of grid spacings {h}")
        dims.append(n)
    return dims


def _maxwell(rng, n, kBT):
    v = rng.normal(0.0, math.sqrt(kBT), size=(n, 3))
    if n:
        v -= v.mean(axis=0)
    return v


def _finish(name, box, phi, h, fpos, spos, kBT, rng, gap=0.0, shuffle_ids=True):
    nf, ns = len(fpos), len(spos)
    pos = np.concatenate([fpos, spos]).astype(np.float32)
    # Clamp any coordinate that rounds up to the box edge in binary32.
    for a in range(3):
        col = pos[:, a]
        col[col >= np.float32(box[a])] = np.nextafter(np.float32(box[a]), np.float32(0))
        col[col < 0] = 0
    vel = np.zeros((nf + ns, 3), np.float64)
    vel[:nf] = _maxwell(rng, nf, kBT)
    types = np.concatenate([np.zeros(nf, np.uint8), np.ones(ns, np.uint8)])
    ids = rng.permutation(nf + ns).astype(np.int32) if shuffle_ids else np.arange(nf + ns, dtype=np.int32)
    # Store in id order so that state arrays index by id.
    order = np.argsort(ids)
    return Workload(name, tuple(float(b) for b in box), phi, h, pos[order],
                    vel[order].astype(np.float32), ids[order], types[order], gap)


def channel(Lx: float, Ly: float, H: float, rho: float = 3.0, layer: float = 1.0,
            kBT: float = 1.0, seed: int = 0, h: float = GRID_H) -> Workload:
    """Plane Poiseuille channel: fluid gap (0, H), solid layers of `layer` r_c."""
    box = (float(Lx), float(Ly), float(H + 2 * layer))
    nx, ny, nz = _grid_dims(box, h)
    z = np.arange(nz) * h
    d = np.where(z <= H, np.minimum(z, H - z), -np.minimum(z - H, box[2] - z))
    phi_z = _phi_from_distance(d)
    phi = np.broadcast_to(phi_z[:, None, None], (nz, ny, nx)).astype(np.float32).copy()
    rng = np.random.default_rng(seed)
    nf = int(round(rho * Lx * Ly * H))
    ns = int(round(rho * Lx * Ly * 2 * layer))
    fz = rng.uniform(0.0, H, size=nf)
    fz[fz == 0.0] = H / 2
    fpos = np.stack([rng.uniform(0, Lx, nf), rng.uniform(0, Ly, nf), fz], axis=1)
    spos = np.stack([rng.uniform(0, Lx, ns), rng.uniform(0, Ly, ns),
                     H + rng.uniform(0.0, 2 * layer, ns)], axis=1)
    return _finish(f"channel_{Lx:g}x{Ly:g}x{H:g}", box, phi, h, fpos, spos, kBT, rng, gap=H)


def keep(w: Workload, mask) -> Workload:
    """The particles of w selected by mask, with ids renumbered 0..m-1 in order."""
    mask = np.asarray(mask, bool)
    m = int(mask.sum())
    return Workload(w.name + "_subset", w.box, w.phi, w.h, w.pos[mask].copy(), w.vel[mask].copy(),
                    np.arange(m, dtype=np.int32), w.type[mask].copy(), w.gap)


def bulk(L, rho: float = 3.0, kBT: float = 1.0, seed: int = 0, h: float = GRID_H) -> Workload:
    """Periodic box of fluid with no solid anywhere (phi = 1)."""
    box = tuple(float(x) for x in (L if np.ndim(L) else (L, L, L)))
    nx, ny, nz = _grid_dims(box, h)
    phi = np.ones((nz, ny, nx), np.float32)
    rng = np.random.default_rng(seed)
    nf = int(round(rho * box[0] * box[1] * box[2]))
    fpos = rng.uniform(0, 1, size=(nf, 3)) * np.asarray(box)
    return _finish(f"bulk_{box[0]:g}x{box[1]:g}x{box[2]:g}", box, phi, h, fpos,
                   np.zeros((0, 3)), kBT, rng)


def _place_spheres(L, nsph, rmin, rmax, rng, max_tries=200000):
    cs, rs = [], []
    tries = 0
    while len(cs) < nsph:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place the requested spheres")
        c = rng.uniform(0, L, 3)
        r = rng.uniform(rmin, rmax)
        ok = True
        for c2, r2 in zip(cs, rs):
            d = c - c2
            d -= L * np.round(d / L)
            if np.linalg.norm(d) < r + r2:
                ok = False
                break
        if ok:
            cs.append(c)
            rs.append(r)
    return np.asarray(cs), np.asarray(rs)


def _sphere_distance(pts, cs, rs, L):
    d = np.full(len(pts), np.inf)
    for c, r in zip(cs, rs):
        dd = pts - c
        dd -= L * np.round(dd / L)
        d = np.minimum(d, np.sqrt((dd * dd).sum(axis=1)) - r)
    return d


def _sphere_distance_two(pts, cs, rs, L):
    """Signed distances to the nearest and the second-nearest sphere surface."""
    d1 = np.full(len(pts), np.inf)
    d2 = np.full(len(pts), np.inf)
    for c, r in zip(cs, rs):
        dd = pts - c
        dd -= L * np.round(dd / L)
        e = np.sqrt((dd * dd).sum(axis=1)) - r
        d2 = np.minimum(d2, np.maximum(d1, e))
        d1 = np.minimum(d1, e)
    return d1, d2


# Beyond this distance from every surface tanh(d / (sqrt(2) eps)) rounds to 1 in binary32.
_PHI_SATURATION_DISTANCE = 7.0


def _sphere_phi(L, cs, rs, h):
    """phi = tanh(d / (sqrt(2) eps)) on the periodic node grid, d the signed distance
    to the union of the spheres.  Each sphere only updates the nodes within
    _PHI_SATURATION_DISTANCE of its surface (every other node rounds to phi = 1 in
    binary32 whatever its distance), with the same arithmetic per node as
    _sphere_distance, so the grid equals the all-spheres evaluation bit for bit."""
    n = int(round(L / h))
    ax = np.arange(n) * h
    dist = np.full((n, n, n), np.inf)  # (z, y, x)
    for c, r in zip(cs, rs):
        reach = r + _PHI_SATURATION_DISTANCE
        sel = []
        for a in range(3):
            lo = int(math.floor((c[a] - reach) / h))
            hi = int(math.ceil((c[a] + reach) / h))
            idx = np.arange(lo, hi + 1) % n if hi - lo + 1 < n else np.arange(n)
            idx = np.unique(idx)
            dd = ax[idx] - c[a]
            dd -= L * np.round(dd / L)
            sel.append((idx, dd * dd))
        (ix, dx2), (iy, dy2), (iz, dz2) = sel
        d = np.sqrt((dx2[None, None, :] + dy2[None, :, None]) + dz2[:, None, None]) - r
        sub = np.ix_(iz, iy, ix)
        dist[sub] = np.minimum(dist[sub], d)
    return _phi_from_distance(dist)


def sphere_pack(L: float, nspheres: int, rmin: float, rmax: float, rho: float = 3.0,
                layer: float = 1.0, kBT: float = 1.0, seed: int = 0,
                h: float = GRID_H) -> Workload:
    """Periodic cube of non-overlapping solid spheres; fluid fills the pores."""
    box = (float(L),) * 3
    rng = np.random.default_rng(seed)
    cs, rs = _place_spheres(L, nspheres, rmin, rmax, rng)
    phi = _sphere_phi(L, cs, rs, h)
    ncand = int(round(rho * L ** 3))
    cand = rng.uniform(0, L, size=(ncand, 3))
    d = np.empty(ncand)
    d2 = np.empty(ncand)
    chunk = 1 << 18
    for s in range(0, ncand, chunk):
        d[s:s + chunk], d2[s:s + chunk] = _sphere_distance_two(cand[s:s + chunk], cs, rs, L)
    # A thin shell 0 < d <= 0.02 r_c next to the curved surfaces stays empty: there the
    # grid-interpolated phase field can fall a little below zero (interpolation error
    # ~ h^2/8 |phi''| ~ 0.012 in phi, ~ 0.009 r_c in distance), and a fluid particle
    # must start on the fluid side of the sharp interface.  Where two surfaces come
    # within ~1 r_c of each other the distance to their union has a ridge, and a grid
    # cell across the ridge interpolates up to ~h/2 below it: points there within
    # 0.15 r_c of a surface stay empty too.
    fpos = cand[(d > 0.02) & ~((d < 0.15) & (d2 < 1.0))]
    spos = cand[(d <= 0) & (d >= -layer)]
    return _finish(f"spheres_{L:g}_{nspheres}", box, phi, h, fpos, spos, kBT, rng)


def ensemble(nsys: int = 64, seed: int = 0, min_fluid: int = 2000, max_fluid: int = 60000,
             edge=(8, 40), gap=(6, 30)):
    """Independent systems of uneven sizes: alternately plane channels (box edges
    and gap widths drawn from `edge` and `gap`) and periodic sphere-pack pores,
    with seeds seed + k and fluid counts kept within [min_fluid, max_fluid]."""
    rng = np.random.default_rng(1_000_003 + seed)
    out = []
    k = 0
    while len(out) < nsys:
        s = seed + k
        k += 1
        if len(out) % 2 == 0:
            H = float(rng.integers(gap[0], gap[1] + 1))
            target = rng.uniform(min_fluid, max_fluid) / (3.0 * H)
            side = max(float(edge[0]), min(float(edge[1]), round(math.sqrt(target))))
            Ly = max(float(edge[0]), min(float(edge[1]), round(target / side)))
            w = channel(side, Ly, H, seed=s)
        else:
            L = float(rng.integers(max(edge[0], 10), min(edge[1], 26) + 1))
            nsph = int(rng.integers(2, 6))
            w = sphere_pack(L, nsph, 0.12 * L, 0.22 * L, seed=s)
        if min_fluid <= w.n_fluid <= max_fluid:
            out.append(w)
    return out


def channel_2d(Lx: float, W: float, rho: float = 4.0, layer: float = 1.0, kBT: float = 1.0,
               seed: int = 0, h: float = GRID_H) -> Workload:
    """Planar channel of width W along y between walls at y = 0 and y = W, as one
    particle layer at z = 1.5 in a box of height 3 (see the module docstring)."""
    box = (float(Lx), float(W + 2 * layer), 3.0)
    nx, ny, nz = _grid_dims(box, h)
    y = np.arange(ny) * h
    d = np.where(y <= W, np.minimum(y, W - y), -np.minimum(y - W, box[1] - y))
    phi_y = _phi_from_distance(d)
    phi = np.broadcast_to(phi_y[None, :, None], (nz, ny, nx)).astype(np.float32).copy()
    rng = np.random.default_rng(seed)
    nf = int(round(rho * Lx * W))
    ns = int(round(rho * Lx * 2 * layer))
    fy = rng.uniform(0.0, W, size=nf)
    fy[fy == 0.0] = W / 2
    fpos = np.stack([rng.uniform(0, Lx, nf), fy, np.full(nf, 1.5)], axis=1)
    spos = np.stack([rng.uniform(0, Lx, ns), W + rng.uniform(0.0, 2 * layer, ns), np.full(ns, 1.5)],
                    axis=1)
    w = _finish(f"channel2d_{Lx:g}x{W:g}", box, phi, h, fpos, spos, kBT, rng, gap=W)
    w.vel[:, 2] = 0.0
    fl = w.type == 0
    if fl.any():
        w.vel[fl, :2] -= w.vel[fl, :2].mean(axis=0)
        # Maxwellian in the plane at k_BT: rescale the two in-plane components
        w.vel[fl, :2] *= np.float32(math.sqrt(kBT) / max(1e-12, float(w.vel[fl, :2].std())))
    return w


def cylinder_2d(L: float, r: float, rho: float = 4.0, layer: float = 1.0, kBT: float = 1.0,
                seed: int = 0, h: float = GRID_H) -> Workload:
    """One disk of radius r centred in a periodic L x L cell (a square array of
    parallel cylinders), as a particle layer at z = 1.5 in a box of height 3."""
    box = (float(L), float(L), 3.0)
    nx, ny, nz = _grid_dims(box, h)
    c = np.array([L / 2, L / 2])
    ax = np.arange(nx) * h
    xx, yy = np.meshgrid(ax, ax, indexing="xy")
    dx = xx - c[0]
    dy = yy - c[1]
    dx -= L * np.round(dx / L)
    dy -= L * np.round(dy / L)
    d2 = np.sqrt(dx * dx + dy * dy) - r
    phi_xy = _phi_from_distance(d2)  # (ny, nx)
    phi = np.broadcast_to(phi_xy[None, :, :], (nz, ny, nx)).astype(np.float32).copy()
    rng = np.random.default_rng(seed)
    ncand = int(round(rho * L * L))
    cand = rng.uniform(0, L, size=(ncand, 2))
    e = cand - c
    e -= L * np.round(e / L)
    d = np.sqrt((e * e).sum(1)) - r
    f2 = cand[d > 0.02]   # see sphere_pack for the empty shell next to curved surfaces
    s2 = cand[(d <= 0) & (d >= -layer)]
    fpos = np.stack([f2[:, 0], f2[:, 1], np.full(len(f2), 1.5)], axis=1)
    spos = np.stack([s2[:, 0], s2[:, 1], np.full(len(s2), 1.5)], axis=1)
    w = _finish(f"cylinder2d_{L:g}_r{r:g}", box, phi, h, fpos, spos, kBT, rng)
    w.vel[:, 2] = 0.0
    fl = w.type == 0
    if fl.any():
        w.vel[fl, :2] -= w.vel[fl, :2].mean(axis=0)
        w.vel[fl, :2] *= np.float32(math.sqrt(kBT) / max(1e-12, float(w.vel[fl, :2].std())))
    return w

