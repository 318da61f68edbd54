"""Statistical observables of the binary32 GPU step against the binary64 oracle.

Trajectories of the two diverge chaotically within a few hundred steps, so they are
compared the way the paper measures a run (Sec. III.A): time averages of the density,
the mean x velocity and the temperature in bins across a driven channel (plane
Poiseuille flow, g_x = 0.05, gap 6), with standard errors from block averages.  Both
start from the same state with the same noise seed; after 2000 steps each samples
8000 steps every 20.  Every bin must agree within 4 combined standard errors.
"""
import numpy as np
import pytest

import oracle
from paper_1807_09896_gb300 import inputs
from parity_helpers import gpu_state, make_system, params_for

pytestmark = pytest.mark.gpu

H, NB, EQUIL, RUN, EVERY, NBLOCK = 6.0, 12, 2000, 8000, 20, 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_09896_gb300 import _build

    _build.build()


def _bin_sums(pos, vel, types):
    """Per bin across the gap: count, sum vx, sum vx^2... for one snapshot."""
    f = types == 0
    z, v = pos[f, 2].astype(np.float64), vel[f].astype(np.float64)
    b = np.floor(z / (H / NB)).astype(np.int64)
    ok = (b >= 0) & (b < NB)
    out = np.zeros((NB, 5))
    for c, val in enumerate((np.ones(ok.sum()), v[ok, 0], v[ok, 1], v[ok, 2], (v[ok] ** 2).sum(1))):
        out[:, c] = np.bincount(b[ok], weights=val, minlength=NB)
    return out


def _observables(sums, nsamples, area):
    n = sums[:, 0]
    rho = n / (nsamples * area * H / NB)
    mv = sums[:, 1:4] / n[:, None]
    T = (sums[:, 4] / n - (mv ** 2).sum(1)) / 3.0
    return np.stack([rho, mv[:, 0], T])  # 3 x NB


def _blocks(snapshots, area):
    per = len(snapshots) // NBLOCK
    obs = [_observables(sum(snapshots[k * per:(k + 1) * per]), per, area) for k in range(NBLOCK)]
    obs = np.array(obs)
    return obs.mean(0), obs.std(0, ddof=1) / np.sqrt(NBLOCK)


def test_profiles_of_binary32_and_binary64_runs_agree_within_errors():
    w = inputs.channel(8.0, 8.0, H, seed=13)
    p = params_for(w, g=(0.05, 0.0, 0.0), seed=4)
    area = w.box[0] * w.box[1]
    # GPU, binary32
    s = make_system(w, p)
    s.step(EQUIL)
    gsnap = []
    for _ in range(RUN // EVERY):
        s.step(EVERY)
        pos, vel, _, types = gpu_state(s)
        gsnap.append(_bin_sums(pos, vel, types))
    s.close()
    # oracle, binary64
    field = oracle.Field(w.phi, w.h)
    st = oracle.State(w.pos.astype(np.float64), w.vel.astype(np.float64), np.zeros((w.n, 3)),
                      w.id.copy(), w.type.copy(), 0)
    st = oracle.init_forces(st, p)
    for _ in range(EQUIL):
        st = oracle.step(st, p, field)
    osnap = []
    for k in range(RUN):
        st = oracle.step(st, p, field)
        if (k + 1) % EVERY == 0:
            osnap.append(_bin_sums(st.pos, st.vel, st.type))
    gm, gs = _blocks(gsnap, area)
    om, os_ = _blocks(osnap, area)
    z = np.abs(gm - om) / np.sqrt(gs ** 2 + os_ ** 2)
    names = ["density", "mean vx", "temperature"]
    for q in range(3):
        print(f"{names[q]:12s} gpu {np.round(gm[q], 3).tolist()}")
        print(f"{'':12s} fp64 {np.round(om[q], 3).tolist()}  max |diff|/sigma {z[q].max():.2f}")
    assert np.all(z < 4.0), z
