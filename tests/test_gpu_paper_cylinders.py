"""Stokes flow through a square array of parallel cylinders (Sec. III.B, Eqs. 20-21).

As in the paper: a 2-D DPD fluid (an exact planar particle layer, see
test_gpu_paper_2d.py) of density 4 with 3120 particle sites in a periodic L x L cell
(L = 28) holding one cylinder, kBT = 0.1, a = 1.875, gamma = 45, sigma = 3, body force
g = 0.005, and the viscosity mu = 3.41 the paper takes from its Poiseuille runs.  The
mean fluid velocity, normalised as 4 pi vbar mu / (rho g L^2), is compared with the
Drummond-Tahir expansion the paper prints as Eq. 20, eps = pi r^2 / L^2 being the solid
area fraction (the paper calls it the void fraction; the constants of Eq. 20 match
the square-array expansion only when eps is the solid fraction).

Measured (one seed, 5 x 10^5 steps of 0.005): eps 0.05 -> 0.784 (Eq. 20: 0.808),
eps 0.1 -> 0.550 (0.507), eps 0.2 -> 0.285 (0.248), eps 0.3 -> 0.165 (0.140); the
paper finds agreement at small eps and fits its own data over all eps by Eq. 21
(0.840, 0.564, 0.332, 0.217 at the same eps).  The test holds the two smallest
fractions to 12% of Eq. 20 and checks the decrease with eps.  FP32 against FP64: the
binary64 oracle ran the same runs (tests/golden/make_fp64_observables.py); the two
means must agree within 4 combined standard errors.
"""
import math
import os

import numpy as np
import pytest

from paper_1807_09896_gb300 import dpd, inputs

pytestmark = pytest.mark.gpu

FP64 = os.path.join(os.path.dirname(__file__), "golden", "fp64_observables.npz")


def eq20(eps):
    """Eq. 20: normalised mean velocity of a square array at solid fraction eps."""
    return (math.log(math.sqrt(math.pi / eps)) + eps - 1.31 - 8.76 * (eps / math.pi) ** 2
            + 63.22 * (eps / math.pi) ** 3)


def eq21(eps):
    """Eq. 21: the paper's fit to its DPD results over all fractions."""
    return math.log(math.sqrt(math.pi / eps)) + 1.7 * eps - 1.31 - 2.15 * eps ** 2 + 1.35 * eps ** 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_09896_gb300 import _build

    _build.build()


def _normalised_mean_velocity(eps, L=28.0, mu=3.41, g=0.005, rho=4.0, kBT=0.1, seed=1):
    r = L * math.sqrt(eps / math.pi)
    w = inputs.cylinder_2d(L, r, kBT=kBT, seed=seed)
    fl = w.type == 0
    w.vel[fl, 0] += np.float32(eq20(eps) * rho * g * L * L / (4 * math.pi * mu))  # head start
    s = dpd.System.from_workload(w, a_ff=1.875, a_fs=1.875, gamma=45.0, sigma=3.0, kBT=kBT,
                                 dt=0.005, g=(g, 0.0, 0.0), rho=rho)
    s.step(100000)
    vs = []
    for _ in range(40):
        s.step(10000)
        st = s.stats()
        vs.append(st[0] / st[4])
    pos = s.state()[0]
    s.close()
    assert np.all(pos[:, 2] == np.float32(1.5))
    return _normalise(np.asarray(vs), L, mu, g, rho)


def _normalise(vs, L=28.0, mu=3.41, g=0.005, rho=4.0):
    """Normalised mean velocity of the samples and its standard error (the samples
    are 50 time units apart, longer than the flow's relaxation time L^2 / (4 pi^2 nu))."""
    f = 4 * math.pi * mu / (rho * g * L * L)
    return f * float(np.mean(vs)), f * float(np.std(vs, ddof=1)) / math.sqrt(len(vs))


@pytest.mark.slow
def test_mean_velocity_through_a_cylinder_array_follows_eq20_at_small_fraction():
    fp64 = np.load(FP64)
    out = {}
    for eps in (0.05, 0.1, 0.2):
        out[eps], err = _normalised_mean_velocity(eps)
        # binary64 oracle, same start, seed and schedule (make_fp64_observables.py)
        v64, err64 = _normalise(fp64[f"cylinders_eps{eps:g}"])
        print(f"eps {eps}: {out[eps]:.4f} +- {err:.4f} (binary64 {v64:.4f} +- {err64:.4f})  "
              f"Eq. 20 {eq20(eps):.4f}  Eq. 21 {eq21(eps):.4f}")
        assert abs(out[eps] - v64) <= 4 * math.hypot(err, err64)
    for eps in (0.05, 0.1):
        assert abs(out[eps] / eq20(eps) - 1.0) < 0.12
    assert out[0.05] > out[0.1] > out[0.2] > 0
