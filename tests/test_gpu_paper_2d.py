"""The paper's 2-D Poiseuille numbers (Sec. III.A, Eqs. 18-19), reproduced on the GPU.

A single layer of particles (all at one z, zero z velocity) in a box three cells high
is an exact 2-D DPD fluid: pair forces lie along the separation, which has no z
component.  The channel of width 10 with 1 r_c solid layers and areal density 4 holds
30 x 12 x 4 = 1440 particles, as in the paper.  The viscosity follows from the
steady profile by Eq. 19 (from the fitted maximum and from the mean), and the
Reynolds number as rho vbar (2a) / mu.

The paper does not state dt or lambda, and its frozen wall particles come from an
equilibrated fluid; over four seeds the values here differ from the printed ones by
2-4% at kBT = 1 (seed spread 2%) and by 0.1-2% at kBT = 0.1 (spread 0.5%).  The bounds
below leave room for one run's statistical error on top.

FP32 against FP64: the binary64 oracle ran each seed's run from the same start on the
same schedule (tests/golden/make_fp64_observables.py); the trajectories separate
(chaos), so the binary32 and binary64 observables must agree within their combined
statistical errors (jackknife over the 6 sampling blocks, 4 sigma).
"""
import os

import numpy as np
import pytest

from flow_analysis import jackknife
from paper_1807_09896_gb300 import dpd, inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_poiseuille_2d.txt")
# binary64 oracle runs of the same starts, seeds and schedules (make_fp64_observables.py)
FP64 = os.path.join(os.path.dirname(__file__), "golden", "fp64_observables.npz")
SEEDS = (0, 1)
BLOCKS = 6


def _rows():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(tuple(float(x) for x in line.split()))
    return out


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_09896_gb300 import _build

    _build.build()


W2D, G2D, RHO2D, NB2D = 10.0, 0.02, 4.0, 100


def _poiseuille_2d(kBT, a, gamma, sigma, dt, seed, mu_guess, Lx=30.0):
    """Block profiles (6 blocks of 100 time units, sampled every 10 steps, 100 bins
    across the channel) after 300 time units from the parabola of mu_guess."""
    W, g, rho = W2D, G2D, RHO2D
    w = inputs.channel_2d(Lx, W, kBT=kBT, seed=seed)
    assert w.n == 1440
    y = w.pos[:, 1].astype(np.float64)
    fl = w.type == 0
    w.vel[fl, 0] += (rho * g * y * (W - y) / (2 * mu_guess))[fl].astype(np.float32)
    s = dpd.System.from_workload(w, a_ff=a, a_fs=a, gamma=gamma, sigma=sigma, kBT=kBT, dt=dt,
                                 g=(g, 0.0, 0.0), rho=rho, seed=seed)
    s.step(int(300.0 / dt))
    s.set_option("sample_every", 10)
    blocks = []
    for _ in range(BLOCKS):
        s.profile(1, NB2D, 0.0, W, mode=3)
        s.step(int(100.0 / dt))
        blocks.append(s.profile(1, NB2D, 0.0, W, mode=2).copy())
    pos = s.state()[0]
    s.close()
    assert np.all(pos[:, 2] == np.float32(1.5))  # the layer stays exactly planar
    return np.array(blocks)


def eq19_observables(prof):
    """mu from the fitted maximum and from the mean velocity (Eq. 19), and Re."""
    W, g, rho = W2D, G2D, RHO2D
    cnt = prof[:, 0]
    u = prof[:, 1] / cnt
    yc = (np.arange(NB2D) + 0.5) * W / NB2D
    inner = (yc > 1.0) & (yc < W - 1.0)
    c2, c1, c0 = np.polyfit(yc[inner], u[inner], 2)
    vmax = c0 - c1 * c1 / (4 * c2)
    vbar = prof[:, 1].sum() / cnt.sum()
    half = W / 2
    mu_max = rho * g * half * half / (2 * vmax)  # Eq. 19, first form
    mu_bar = rho * g * half * half / (3 * vbar)  # Eq. 19, second form
    return np.array([mu_max, mu_bar, rho * vbar * W / mu_max])


def _with_errors(blocks):
    return jackknife(lambda keep: eq19_observables(blocks[keep].sum(axis=0)), len(blocks))


@pytest.mark.slow
@pytest.mark.parametrize("row", _rows(), ids=["kBT=1", "kBT=0.1"])
def test_printed_viscosity_and_reynolds_number(row):
    kBT, a, gamma, sigma, mu_max_p, mu_bar_p, re_p = row
    dt = 0.01 if kBT >= 1.0 else 0.005  # gamma = 45 needs the smaller step
    fp64 = np.load(FP64)
    runs, errs = [], []
    for seed in SEEDS:
        blocks = _poiseuille_2d(kBT, a, gamma, sigma, dt, seed, mu_guess=mu_bar_p)
        (obs, err) = _with_errors(blocks)
        # the binary64 oracle from the same start, seed and schedule
        (obs64, err64) = _with_errors(fp64[f"poiseuille2d_kBT{kBT:g}_seed{seed}"])
        print(f"kBT {kBT} seed {seed}: (mu(vmax), mu(vbar), Re) binary32 {obs} +- {err}, "
              f"binary64 {obs64} +- {err64}")
        assert np.all(np.abs(obs - obs64) <= 4 * np.hypot(err, err64))
        runs.append(obs)
        errs.append(err)
    mu_max, mu_bar, re = np.mean(runs, axis=0)
    print(f"kBT {kBT}: mu(vmax) {mu_max:.4f} (paper {mu_max_p}), mu(vbar) {mu_bar:.4f} "
          f"(paper {mu_bar_p}), Re {re:.2f} (paper {re_p})")
    tol = 0.08 if kBT >= 1.0 else 0.04
    assert abs(mu_max / mu_max_p - 1.0) < tol
    assert abs(mu_bar / mu_bar_p - 1.0) < tol
    assert abs(re / re_p - 1.0) < 2 * tol
    # Eq. 19's two estimates agree for a parabolic profile with no slip
    assert abs(mu_max / mu_bar - 1.0) < 0.04
