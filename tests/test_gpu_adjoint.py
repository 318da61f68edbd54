"""Gradients of a near-wall velocity-profile loss with respect to (a_fs, gamma, g_x)
from the hand-written adjoint, against central differences of the FP64 oracle.

The loss bins fluid particles by distance to the nearer wall (8 bins of 0.25 r_c)
and compares the window-averaged x velocity of each bin with the no-slip Poiseuille
parabola (Eq. 18).  The noise stream is fixed (same seed and step counter), and the
finite differences keep the events of the base trajectory frozen, as the adjoint
does: the reflection decisions of the +h and -h runs are checked to equal the base
run's (h shrinks until they do), and bin membership is taken from the base run.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1807_09896_gb300 import adjoint, dpd, inputs
from parity_helpers import gpu_state, make_system, params_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_09896_gb300 import _build

    _build.build()


def _bins(pos, types, loss):
    x = pos[:, loss.axis].astype(np.float32)
    d = np.minimum(x - np.float32(loss.wall_lo), np.float32(loss.wall_hi) - x)
    b = np.floor(d * np.float32(1.0 / loss.width))
    ok = (d >= 0) & (b < loss.nbins) & (types == 0)
    return np.where(ok, b, -1).astype(np.int64)


def _oracle_run(w, p, nsteps):
    field = oracle.Field(w.phi, w.h)
    s = oracle.State(w.pos.astype(np.float64), w.vel.astype(np.float64), np.zeros((w.n, 3)),
                     w.id.copy(), w.type.copy(), 0)
    s = oracle.init_forces(s, p)
    traj = []
    for _ in range(nsteps):
        s, refl = oracle.step(s, p, field, return_reflected=True)
        traj.append((s.pos.copy(), s.vel[:, 0].copy(), refl))
    return traj


def _frozen_loss(traj, members, loss):
    sums = np.zeros(loss.nbins)
    cnt = np.zeros(loss.nbins)
    for (_, vx, _), b in zip(traj, members):
        ok = b >= 0
        np.add.at(sums, b[ok], vx[ok])
        np.add.at(cnt, b[ok], 1.0)
    m = cnt > 0
    u = sums[m] / cnt[m]
    return float(((u - loss.target[m]) ** 2).sum())


def _params(w, theta, seed):
    a_fs, gamma, gx = theta
    return params_for(w, g=(gx, 0.0, 0.0), seed=seed, a_fs=a_fs, gamma=gamma,
                      sigma=math.sqrt(2.0 * gamma * 1.0))


def oracle_fd_gradient(w, theta, loss, nsteps, seed, rel_h=(1e-4, 1e-4, 1e-3)):
    """Central differences of the FP64 oracle's loss with frozen events."""
    base = _oracle_run(w, _params(w, theta, seed), nsteps)
    members = [_bins(pos, w.type, loss) for pos, _, _ in base]
    L0 = _frozen_loss(base, members, loss)
    grad = np.zeros(3)
    for k in range(3):
        h = rel_h[k] * abs(theta[k])
        for _ in range(4):
            runs = []
            for sgn in (1.0, -1.0):
                t = list(theta)
                t[k] += sgn * h
                runs.append(_oracle_run(w, _params(w, t, seed), nsteps))
            same = all(np.array_equal(a[2], b[2]) and np.array_equal(a[2], c[2])
                       for a, b, c in zip(base, runs[0], runs[1]))
            if same:
                break
            h /= 4.0
        assert same, f"reflection decisions still differ at h = {h}"
        grad[k] = (_frozen_loss(runs[0], members, loss) - _frozen_loss(runs[1], members, loss)) / (2 * h)
    return L0, grad


def _setup(Lx=8.0, Ly=6.0, H=6.0, seed=31, theta=(25.0, 4.5, 0.05)):
    w = inputs.channel(Lx, Ly, H, seed=seed)
    target = adjoint.poiseuille_wall_target(H, theta[2], 3.0, 0.9, 8, 0.25)
    loss = adjoint.NearWallLoss(0.0, H, target)
    p = _params(w, theta, seed)
    s = make_system(w, p)
    return w, s, loss


def _reset(s, w):
    s.set_option("step", 0)
    s.set_particles(w.pos4(), w.vel4(), w.id, w.type)


def test_adjoint_gradient_matches_oracle_finite_differences_20_steps():
    theta = (25.0, 4.5, 0.05)
    w, s, loss = _setup(theta=theta)
    L, g = adjoint.window_loss_and_grad(s, theta, loss, nsteps=20, ckpt_every=5)
    L0, g_fd = oracle_fd_gradient(w, theta, loss, 20, seed=31)
    assert abs(L - L0) <= 1e-4 * abs(L0) + 1e-12, (L, L0)
    for k, name in enumerate(["a_fs", "gamma", "g_x"]):
        assert abs(g[k] - g_fd[k]) <= 2e-3 * abs(g_fd[k]) + 1e-9 * abs(L0), (name, g[k], g_fd[k])
    s.close()


def test_checkpoint_interval_does_not_change_the_gradient():
    theta = (30.0, 4.0, 0.05)
    w, s, loss = _setup(theta=theta, seed=32)
    out = []
    for ck in (4, 8, 16):
        _reset(s, w)
        out.append(adjoint.window_loss_and_grad(s, theta, loss, nsteps=16, ckpt_every=ck))
    for L, g in out[1:]:
        assert abs(L - out[0][0]) <= 1e-12 * abs(out[0][0])
        np.testing.assert_allclose(g, out[0][1], rtol=1e-9, atol=0)
    s.close()


def test_whole_window_record_and_segment_recompute_give_the_same_gradient():
    """The reverse pass walks the same recorded steps whether the forward pass kept the
    whole window's record (it fits the default budget) or only checkpoints from which
    each segment is recomputed (budget 0): same loss and gradient, bit for bit.  A
    repeated call (the workspace is reused) gives the same bits too: the sums do not
    depend on the order the warps add in."""
    theta = (25.0, 4.5, 0.05)
    w, s, loss = _setup(theta=theta, seed=36)
    out = []
    for budget in (2048.0, None, 0.0, None):
        _reset(s, w)
        if budget is not None:
            s.set_option("adjoint_tape_mb", budget)
        out.append(adjoint.window_loss_and_grad(s, theta, loss, nsteps=24, ckpt_every=6))
    for o in out[1:]:
        assert o[0] == out[0][0]
        np.testing.assert_array_equal(o[1], out[0][1])
    s.close()


def test_window_leaves_the_state_a_plain_step_leaves():
    theta = (25.0, 4.5, 0.05)
    w, s, loss = _setup(theta=theta, seed=33)
    before = s.stats()
    adjoint.window_loss_and_grad(s, theta, loss, nsteps=12, ckpt_every=4)
    after_window = gpu_state(s)
    window = s.stats() - before  # counters are cumulative: compare what the call added
    _reset(s, w)
    before = s.stats()
    s.step(12)
    for x, y in zip(after_window, gpu_state(s)):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(window[5:7], (s.stats() - before)[5:7])
    assert s.stats()[7] == 12
    s.close()


def test_autograd_function_returns_the_adjoint_gradient():
    import torch

    theta0 = (25.0, 4.5, 0.05)
    w, s, loss = _setup(theta=theta0, seed=34)
    theta = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    L = adjoint.DPDWindow().apply(theta, s, loss, 10, 5)
    (3.0 * L).backward()
    _reset(s, w)
    L2, g = adjoint.window_loss_and_grad(s, theta0, loss, 10, 5)
    assert abs(float(L.detach()) - L2) <= 1e-12 * abs(L2)
    np.testing.assert_allclose(theta.grad.numpy(), 3.0 * g, rtol=1e-12)
    s.close()


def _c5():
    theta = (25.0, 4.5, 0.02)
    w = inputs.channel(32.0, 16.0, 16.0, seed=0)
    target = adjoint.poiseuille_wall_target(16.0, theta[2], 3.0, 0.9, 8, 0.25)
    loss = adjoint.NearWallLoss(0.0, 16.0, target)
    return theta, w, loss


@pytest.mark.slow
def test_adjoint_on_the_32x16x16_channel_over_100_steps():
    """The calibration workload (~25k fluid particles) with a checkpoint every 20
    steps: over 100 steps the adjoint agrees with the oracle's central differences
    to 1% (measured: 0.3% for a_fs, 0.1% for gamma, 1e-5 for g_x)."""
    theta, w, loss = _c5()
    s = make_system(w, _params(w, theta, 0))
    L, g = adjoint.window_loss_and_grad(s, theta, loss, nsteps=100, ckpt_every=20)
    L0, g_fd = oracle_fd_gradient(w, theta, loss, 100, seed=0, rel_h=(1e-7, 1e-7, 1e-6))
    assert abs(L - L0) <= 1e-4 * abs(L0)
    for k in range(3):
        assert abs(g[k] - g_fd[k]) <= 1e-2 * abs(g_fd[k]) + 1e-9 * abs(L0), (k, g, g_fd)
    s.close()


def test_adjoint_rejects_walls_sliding_at_different_velocities():
    w, s, loss = _setup(seed=35)
    s.set_option("shear_x", 0.05)
    with pytest.raises(dpd.DPDError):
        adjoint.window_loss_and_grad(s, (25.0, 4.5, 0.05), loss, nsteps=4, ckpt_every=2)
    s.close()
