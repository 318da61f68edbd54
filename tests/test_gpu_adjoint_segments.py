"""The 200-step adjoint window of the calibration channel (32 x 16 x 16 r_c, ~25k fluid
particles, a checkpoint every 20 steps) checked segment by segment against the FP64
oracle (Eqs. 4-10 and 17, differentiated).

Over 200 steps one noise realization is chaotic: the binary32 and binary64 trajectories
separate and so do their whole-window gradients, which says nothing about whether the
adjoint is right.  So the window is split where the library splits it.  For segment k
the oracle starts from the GPU's own checkpoint s_k and runs the segment's 20 steps;
the scalar

    J_k(theta, s) = <lambda_{k+1}, state after the segment> + sum of the loss terms of
                    the segment's inner states (linearised: coef_b * vx summed over
                    bin b, with the GPU's coef),

with lambda_{k+1} the GPU's adjoint of the segment's end state, has central
differences (events frozen: reflection decisions checked equal, bins taken from the
oracle's base run) that must equal the GPU's share of dL/dtheta accumulated while
reversing segment k (to 2e-3 of itself or 1e-4 of the largest segment share), and,
along a random direction of the start state, the GPU's adjoint lambda_k (to 2e-3 of
the derivative or 1e-4 of the sum of the absolute terms it adds up, which cancel to a
small total in the later segments; the binary32 adjoint of 20 steps measured up to
3.3e-5 of that sum).  The whole-window gradient is then the sum of these checked pieces
(asserted too), and the binary32-vs-binary64 difference of the whole-window gradient
is stated for the record.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1807_09896_gb300 import adjoint, dpd, inputs
from parity_helpers import make_system, params_for

pytestmark = pytest.mark.gpu

THETA = (25.0, 4.5, 0.02)
NSTEPS, K = 200, 20
SEED = 0
REL_TOL = 2e-3


@pytest.fixture(scope="module")
def window():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_09896_gb300 import _build

    _build.build()
    w = inputs.channel(32.0, 16.0, 16.0, seed=SEED)
    target = adjoint.poiseuille_wall_target(16.0, THETA[2], 3.0, 0.9, 8, 0.25)
    loss = adjoint.NearWallLoss(0.0, 16.0, target)
    s = make_system(w, _params(w, THETA))
    adjoint.set_theta(s, THETA)
    L, g, rec = dpd.dpd_adjoint_window_record(s.h, NSTEPS, K, loss.axis, loss.wall_lo, loss.wall_hi,
                                              loss.target, loss.width, True)
    s.close()
    return w, loss, L, g, rec


def _params(w, theta):
    a_fs, gamma, gx = theta
    return params_for(w, g=(gx, 0.0, 0.0), seed=SEED, a_fs=a_fs, gamma=gamma,
                      sigma=math.sqrt(2.0 * gamma * 1.0))


def _bins(pos, types, loss):
    x = pos[:, loss.axis].astype(np.float32)
    d = np.minimum(x - np.float32(loss.wall_lo), np.float32(loss.wall_hi) - x)
    b = np.floor(d * np.float32(1.0 / loss.width))
    ok = (d >= 0) & (b < loss.nbins) & (types == 0)
    return np.where(ok, b, -1).astype(np.int64)


def _segment_run(w, theta, start, step0, recompute_force):
    """K oracle steps from the state `start` = (pos, vel, frc); returns the states after
    every step and the reflection flags."""
    p = _params(w, theta)
    field = oracle.Field(w.phi, w.h)
    pos, vel, frc = (a.astype(np.float64) for a in start)
    st = oracle.State(pos.copy(), vel.copy(), frc.copy(), w.id.copy(), w.type.copy(), step0)
    if recompute_force:  # the window's first force is computed with the parameters
        st = oracle.init_forces(st, p)
    out = []
    for _ in range(K):
        st, refl = oracle.step(st, p, field, return_reflected=True)
        out.append((st.pos.copy(), st.vel.copy(), st.frc.copy(), refl))
    return out


def _J(run, lam_end, members, coef, start_vel=None, start_members=None):
    pos, vel, frc, _ = run[-1]
    J = float((lam_end[:, 0, :3] * pos).sum() + (lam_end[:, 1, :3] * vel).sum() +
              (lam_end[:, 2, :3] * frc).sum())
    for (_, v, _, _), b in zip(run[:-1], members[:-1]):
        ok = b >= 0
        J += float((coef[b[ok]] * v[ok, 0]).sum())
    if start_vel is not None:  # the start state's own loss term (it is part of lambda_k)
        ok = start_members >= 0
        J += float((coef[start_members[ok]] * start_vel[ok, 0]).sum())
    return J


def _same_events(a, b):
    return all(np.array_equal(x[3], y[3]) for x, y in zip(a, b))


def _segment_checks(w, loss, rec, k):
    ck = rec["ckpt"][k]
    start = (ck[:, 0, :3], ck[:, 1, :3], ck[:, 2, :3])
    step0 = int(rec["seg_step"][k])
    lam_end = rec["adj"][k + 1].astype(np.float64)
    coef = rec["coef"].astype(np.float64)
    first = k == 0
    base = _segment_run(w, THETA, start, step0, first)
    members = [_bins(r[0], w.type, loss) for r in base]
    # parameters
    fd = np.zeros(3)
    for j, rel in enumerate((1e-5, 1e-5, 1e-4)):
        h = rel * abs(THETA[j])
        for _ in range(6):
            runs = []
            for sgn in (1.0, -1.0):
                t = list(THETA)
                t[j] += sgn * h
                runs.append(_segment_run(w, t, start, step0, first))
            if _same_events(base, runs[0]) and _same_events(base, runs[1]):
                break
            h /= 4.0
        assert _same_events(base, runs[0]) and _same_events(base, runs[1])
        fd[j] = (_J(runs[0], lam_end, members, coef) - _J(runs[1], lam_end, members, coef)) / (2 * h)
    # the start state along a random direction (fluid particles), for k >= 1 (the
    # window's first force is recomputed from positions and velocities)
    state = None
    if not first:
        rng = np.random.default_rng(100 + k)
        fl = (w.type == 0)[:, None]
        dirs = [rng.normal(size=a.shape) * fl for a in start]
        lam_k = rec["adj"][k].astype(np.float64)
        predicted = sum(float((lam_k[:, q, :3] * dirs[q]).sum()) for q in range(3))
        # the scale of the terms of that sum (they cancel to a small total in places)
        terms = sum(float(np.abs(lam_k[:, q, :3] * dirs[q]).sum()) for q in range(3))
        smem = _bins(start[0], w.type, loss)
        h = 1e-6
        for _ in range(6):
            vals, runs = [], []
            for sgn in (1.0, -1.0):
                st = tuple(a.astype(np.float64) + sgn * h * d for a, d in zip(start, dirs))
                r = _segment_run(w, THETA, st, step0, False)
                runs.append(r)
                vals.append(_J(r, lam_end, members, coef, st[1], smem))
            if _same_events(base, runs[0]) and _same_events(base, runs[1]):
                break
            h /= 4.0
        assert _same_events(base, runs[0]) and _same_events(base, runs[1])
        state = (predicted, (vals[0] - vals[1]) / (2 * h), terms)
    return fd, state


def test_segment_vjps_match_oracle_central_differences(window):
    w, loss, L, g, rec = window
    nseg = NSTEPS // K
    fds, states = [], []
    for k in range(nseg):
        fd, state = _segment_checks(w, loss, rec, k)
        fds.append(fd)
        states.append(state)
        print(f"segment {k}: gpu {rec['seg_grad'][k]}, oracle fd {fd}"
              + (f"; state direction gpu {state[0]:.6e} oracle fd {state[1]:.6e} (terms "
                 f"{state[2]:.3e})" if state else ""))
    fds = np.array(fds)
    scale = np.abs(fds).max(axis=0)
    for k in range(nseg):
        err = np.abs(rec["seg_grad"][k] - fds[k])
        assert np.all(err <= REL_TOL * np.abs(fds[k]) + 1e-4 * scale), (k, rec["seg_grad"][k], fds[k])
        if states[k] is not None:
            pred, fd, terms = states[k]
            assert abs(pred - fd) <= REL_TOL * abs(fd) + 1e-4 * terms, (k, pred, fd, terms)
    # the whole-window gradient is the sum of the checked segment shares
    np.testing.assert_allclose(rec["seg_grad"].sum(axis=0), g, rtol=1e-9, atol=1e-12 * np.abs(g).max())


def test_whole_window_fp32_against_fp64_is_stated(window):
    """The binary32 window gradient against central differences of the binary64 window
    (same start, same noise): stated, not asserted beyond the loss."""
    from test_gpu_adjoint import oracle_fd_gradient

    w, loss, L, g, rec = window
    L0, g_fd = oracle_fd_gradient(w, THETA, loss, NSTEPS, seed=SEED, rel_h=(1e-7, 1e-7, 1e-6))
    print(f"200-step window: loss binary32 {L:.6e} binary64 {L0:.6e}; dL/d(a_fs, gamma, g_x) "
          f"binary32 adjoint {g}, binary64 central differences {g_fd}")
    assert abs(L - L0) <= 1e-3 * abs(L0)
    assert np.all(np.isfinite(g))
