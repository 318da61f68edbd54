"""Closed-form channel flows and block statistics used by the flow tests (test code).

Plane Poiseuille flow driven by a body force g (acceleration along x) between walls
at z = -b and z = H + b (b: slip length; b = 0 is the no-slip wall at the phi = 0
planes z = 0 and z = H), kinematic viscosity nu:

* steady (Eq. 18):  u(z) = g zeta (H' - zeta) / (2 nu),  zeta = z + b, H' = H + 2 b;
* start-up from rest: u(z, t) = steady(z) - sum_{n odd} 4 g H'^2 / (nu pi^3 n^3)
  sin(n pi zeta / H') exp(-nu n^2 pi^2 t / H'^2), the Fourier series of the steady
  parabola (zeta (H' - zeta) = sum_{n odd} 8 H'^2 / (pi^3 n^3) sin(n pi zeta / H'))
  relaxing mode by mode under u_t = nu u_zz + g;
* from a parabola of another viscosity nu0: the same modes with amplitude
  (1/nu0 - 1/nu) instead of -1/nu.

Binned profiles are compared with the model averaged over each bin (Gauss-Legendre)
and over the sample times of each block.  Error bars: jackknife over blocks.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import least_squares

_GL_X, _GL_W = np.polynomial.legendre.leggauss(5)


def _modes(zeta, t, nu, Hp, nmax):
    n = np.arange(1, nmax + 1, 2, dtype=np.float64)
    s = np.sin(np.pi * np.outer(zeta, n) / Hp)                       # (z, n)
    e = np.exp(-nu * (np.pi * n / Hp) ** 2 * np.asarray(t)[:, None])  # (t, n)
    c = 4.0 * Hp * Hp / (np.pi ** 3 * n ** 3)
    return (s * c) @ e.mean(axis=0)


def channel_velocity(z, times, g, nu, H, b, nu0=None, nmax=401):
    """Mean over `times` of u(z, t) for flow started at t = 0 from rest (nu0 None) or
    from the steady parabola of viscosity nu0 (no slip at the effective walls)."""
    Hp = H + 2.0 * b
    zeta = np.asarray(z, np.float64) + b
    steady = g * zeta * (Hp - zeta) / (2.0 * nu)
    amp = -g / nu if nu0 is None else g * (1.0 / nu0 - 1.0 / nu)
    return steady + amp * _modes(zeta, times, nu, Hp, nmax)


def bin_average(fn, lo, width, nbins):
    """Average of fn(z) over each of nbins bins of `width` starting at lo."""
    c = lo + (np.arange(nbins) + 0.5) * width
    z = c[:, None] + 0.5 * width * _GL_X[None, :]
    vals = fn(z.ravel()).reshape(z.shape)
    return (vals * _GL_W[None, :]).sum(axis=1) / 2.0


def fit_channel(u_blocks, block_times, mask, g, H, lo, width, x0=(0.3, 0.0), nu0=None):
    """Least-squares (nu, b) of the binned mean velocities u_blocks[k, bin] (bins in
    `mask`) against the model averaged over block k's sample times."""
    nbins = u_blocks.shape[1]

    def resid(x):
        nu, b = x
        r = []
        for u, t in zip(u_blocks, block_times):
            m = bin_average(lambda z: channel_velocity(z, t, g, nu, H, b, nu0), lo, width, nbins)
            r.append((u - m)[mask])
        return np.concatenate(r)

    sol = least_squares(resid, np.asarray(x0, np.float64), x_scale=(0.1, 0.1))
    return sol.x, resid(sol.x)


def jackknife(estimate, nblocks):
    """Jackknife mean and standard error of estimate(blocks kept) over nblocks blocks."""
    full = np.asarray(estimate(np.arange(nblocks)), np.float64)
    parts = np.array([estimate(np.delete(np.arange(nblocks), k)) for k in range(nblocks)],
                     np.float64)
    mean = parts.mean(axis=0)
    err = np.sqrt((nblocks - 1) / nblocks * ((parts - mean) ** 2).sum(axis=0))
    return full, err


def profile_fields(prof, samples, area, width, rho_ref=None):
    """Per-bin density, mean x velocity and temperature from the library's profile sums
    {count, sum vx, sum vy, sum vz, sum |v|^2} accumulated over `samples` samples."""
    cnt = prof[:, 0]
    safe = np.maximum(cnt, 1.0)
    u = prof[:, 1:4] / safe[:, None]
    dens = cnt / (samples * area * width)
    temp = (prof[:, 4] / safe - (u * u).sum(axis=1)) / 3.0
    if rho_ref is not None:
        dens = dens / rho_ref
    return dens, u[:, 0], temp


def parabola_fit(zc, u, mask):
    """Least-squares parabola through (zc, u) on mask: its maximum, its zeros, and the
    coefficients (c2, c1, c0)."""
    c2, c1, c0 = np.polyfit(zc[mask], u[mask], 2)
    disc = np.sqrt(max(c1 * c1 - 4 * c2 * c0, 0.0))
    z0, z1 = sorted(((-c1 - disc) / (2 * c2), (-c1 + disc) / (2 * c2)))
    return c0 - c1 * c1 / (4 * c2), (z0, z1), (c2, c1, c0)
