"""Gradient-based calibration of the wall interaction: a ``torch.autograd.Function``
over a window of DPD time steps whose backward pass is the library's hand-written
adjoint (``dpd_adjoint_window`` in include/dpd.h).

The loss compares the near-wall velocity profile of a channel with a target
profile, e.g. the no-slip Poiseuille parabola of Eq. 18 (Sec. III.A).  The
parameters are theta = (a_fs, gamma, g_x): the fluid-solid conservative amplitude
of Eq. 4, the dissipative coefficient of Eq. 6 (with sigma = sqrt(2 gamma kBT),
Eq. 8, kept tied by default) and the body force.  The forward call runs the window
and the adjoint at once; backward only scales the stored gradient.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import dpd


def poiseuille_wall_target(H: float, g_x: float, rho: float, mu: float, nbins: int,
                           width: float) -> np.ndarray:
    """No-slip plane Poiseuille velocity (Eq. 18 with y measured from the centre)
    at the centres of near-wall bins: u(d) = rho g d (H - d) / (2 mu), d the
    distance to the wall."""
    d = (np.arange(nbins) + 0.5) * width
    return rho * g_x * d * (H - d) / (2.0 * mu)


@dataclass
class NearWallLoss:
    """Bins of width `width` by distance to the nearer of the walls at wall_lo and
    wall_hi along `axis`; L = sum_b (mean vx in bin b over the window - target_b)^2."""

    wall_lo: float
    wall_hi: float
    target: np.ndarray
    width: float = 0.25
    axis: int = 2

    @property
    def nbins(self) -> int:
        return len(self.target)


def set_theta(system, theta):
    """Write (a_fs, gamma, g_x) into a System.  With tie_sigma the library itself
    sets sigma from gamma (Eq. 8) when the window starts."""
    a_fs, gamma, g_x = (float(x) for x in theta)
    system.set_option("a_fs", a_fs)
    system.set_option("gamma", gamma)
    system.set_option("g_x", g_x)


def window_loss_and_grad(system, theta, loss: NearWallLoss, nsteps: int, ckpt_every: int,
                         tie_sigma: bool = True):
    """Set theta, run the window on the GPU, return (L, dL/dtheta)."""
    set_theta(system, theta)
    return dpd.dpd_adjoint_window(system.h, nsteps, ckpt_every, loss.axis, loss.wall_lo,
                                  loss.wall_hi, loss.target, loss.width, tie_sigma)


def _autograd_function():
    import torch

    class DPDWindow(torch.autograd.Function):
        """L(theta) over a window of steps of `system`; theta = (a_fs, gamma, g_x)."""

        @staticmethod
        def forward(ctx, theta, system, loss, nsteps, ckpt_every, tie_sigma=True):
            L, g = window_loss_and_grad(system, theta.detach().cpu().double().numpy(), loss,
                                        nsteps, ckpt_every, tie_sigma)
            ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
            return theta.new_tensor(L)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g, None, None, None, None, None

    return DPDWindow


_cache = {}


def DPDWindow():
    """The autograd Function class (built on first use so torch is imported lazily)."""
    if "f" not in _cache:
        _cache["f"] = _autograd_function()
    return _cache["f"]
