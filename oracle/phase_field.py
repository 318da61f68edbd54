"""FP64 oracle of the phase-field relaxation of Sec. II.B (Eqs. 13-15).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Starting from a step function (phi = +1 in the fluid, -1 in the solid) the phase
field is relaxed in pseudo time t' = t / tau on a periodic grid of spacing h, in the
scaled coordinates x' = x / eps:

    d phi / dt' = lap' phi + phi (1 - phi^2) - kappa |grad' phi|,
    kappa = div'(grad' phi / |grad' phi|)                            (Eq. 15)

Written out, kappa |grad phi| = lap phi - phi_nn, with phi_nn = n . H n the second
derivative along the unit normal n = grad phi / |grad phi| and H the Hessian, so the
right-hand side is phi_nn + phi (1 - phi^2): the one-dimensional Allen-Cahn equation
(Eq. 13) along the normal, whose steady profile is Eq. 14, tanh(d / (sqrt(2) eps)).
Without the curvature term (curvature=False) the right-hand side is that of Eq. 13
in every direction, and curved interfaces move (a sphere shrinks).

The normal is undefined where grad phi = 0 (the centre of a blob, a saddle between
two), and near such points its direction is ill-conditioned.  Reading R15: the second
derivative along the normal is blended into the Laplacian there,

    phi_nn = (n.H.n |grad phi|^2 + delta lap phi) / (|grad phi|^2 + delta),

delta = 1e-4 in scaled units.  On an interface |grad' phi|^2 >= 0.02 within 2 eps of
phi = 0 (0.5 at phi = 0), so the curvature term changes by less than 0.5% there;
far from interfaces phi is flat and both forms vanish.

Discretisation (the CUDA solver uses the same formulas in binary32): second-order
central differences for the gradient, the pure and the mixed second derivatives;
explicit Euler steps of dtau.  Arrays are indexed [z, y, x].
"""
from __future__ import annotations

import numpy as np

DELTA = 1e-4  # blend of the normal second derivative into the Laplacian where grad phi -> 0


def _d(phi, axis, k):
    return np.roll(phi, -k, axis=axis)


def rhs(phi: np.ndarray, h: float, eps: float, curvature: bool = True) -> np.ndarray:
    """Right-hand side of Eq. 15 (curvature=True) or Eq. 13 (False) at every node."""
    inv = eps / h  # 1 / h' with h' = h / eps
    ax = {"x": 2, "y": 1, "z": 0}
    p = phi
    g = {}
    s2 = {}
    for c, a in ax.items():
        g[c] = (_d(p, a, 1) - _d(p, a, -1)) * (0.5 * inv)
        s2[c] = (_d(p, a, 1) - 2.0 * p + _d(p, a, -1)) * (inv * inv)
    mixed = {}
    for c1, c2 in (("x", "y"), ("x", "z"), ("y", "z")):
        a1, a2 = ax[c1], ax[c2]
        pp = np.roll(np.roll(p, -1, a1), -1, a2)
        pm = np.roll(np.roll(p, -1, a1), 1, a2)
        mp = np.roll(np.roll(p, 1, a1), -1, a2)
        mm = np.roll(np.roll(p, 1, a1), 1, a2)
        mixed[c1 + c2] = (pp - pm - mp + mm) * (0.25 * inv * inv)
    lap = s2["x"] + s2["y"] + s2["z"]
    reaction = p * (1.0 - p * p)
    if not curvature:
        return lap + reaction
    g2 = g["x"] ** 2 + g["y"] ** 2 + g["z"] ** 2
    num = (g["x"] ** 2 * s2["x"] + g["y"] ** 2 * s2["y"] + g["z"] ** 2 * s2["z"]
           + 2.0 * (g["x"] * g["y"] * mixed["xy"] + g["x"] * g["z"] * mixed["xz"]
                    + g["y"] * g["z"] * mixed["yz"]))
    phi_nn = (num + DELTA * lap) / (g2 + DELTA)
    return phi_nn + reaction


def relax(phi0: np.ndarray, h: float, eps: float, iters: int, dtau: float,
          curvature: bool = True) -> np.ndarray:
    """`iters` explicit Euler steps of Eq. 15 (or Eq. 13) from phi0."""
    phi = np.asarray(phi0, dtype=np.float64).copy()
    for _ in range(iters):
        phi = phi + dtau * rhs(phi, h, eps, curvature)
    return phi
