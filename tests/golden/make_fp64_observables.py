"""Writes fp64_observables.npz: the FP64 oracle's binned statistics for the runs whose
binary32 GPU results the tests report, from the same start, seed and schedule, so that
the FP32-vs-FP64 difference of each reported observable can be stated with error bars.

Runs (each reproduces a GPU test's schedule step for step; see those tests):

* poiseuille2d_kBT{1,0.1}_seed{0,1}: the planar channel of Sec. III.A (width 10, 1440
  particles, density 4), 300 time units from the parabola of the printed viscosity,
  then 600 time units sampled every 10 steps in 6 blocks of 100 bins across the
  channel (tests/test_gpu_paper_2d.py);
* cylinders_eps{0.05,0.1,0.2}: the square cylinder array of Sec. III.B (L = 28), 10^5
  steps, then 40 samples of the mean fluid velocity, one every 10^4 steps
  (tests/test_gpu_paper_cylinders.py);
* channel_slice_{startup,parabola}: a 16 x 8 slice of the 32-gap channel (g_x 0.01),
  10 blocks of 1000 steps sampled every 10 steps in 64 bins across the gap, from rest
  and from the parabola of kinematic viscosity 0.295 (tests/test_gpu_channel_c2.py).

Only the oracle (and the seeded input generators) run here.  Usage:
    python tests/golden/make_fp64_observables.py [--jobs J] [--only NAME ...]
"""
from __future__ import annotations

import argparse
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "fp64_observables.npz")

# run parameters shared with the GPU tests (they import these)
POISEUILLE_2D = {  # kBT: (a, gamma, sigma, dt, printed mu from the mean velocity)
    1.0: (18.75, 4.5, 3.0, 0.01, 0.912),
    0.1: (1.875, 45.0, 3.0, 0.005, 3.4066),
}
POISEUILLE_2D_SEEDS = (0, 1)
POISEUILLE_2D_BLOCKS = 6
CYLINDER_EPS = (0.05, 0.1, 0.2)
SLICE = (16.0, 8.0, 32.0, 0.01)  # Lx, Ly, gap, g_x
SLICE_NU0 = 0.295
SLICE_BLOCKS, SLICE_BLOCK_STEPS, SLICE_EVERY, SLICE_NB = 10, 1000, 10, 64


def eq20(eps):
    """Eq. 20 (the cylinder runs start from its mean velocity)."""
    return (math.log(math.sqrt(math.pi / eps)) + eps - 1.31 - 8.76 * (eps / math.pi) ** 2
            + 63.22 * (eps / math.pi) ** 3)


def _setup():
    sys.path.insert(0, ROOT)
    import oracle
    from oracle import build

    build.build()
    return oracle


def _state(oracle, w, vel=None):
    v = w.vel if vel is None else vel
    return oracle.State(w.pos.astype(np.float64), np.asarray(v, np.float32)[:, :3].astype(np.float64),
                        np.zeros((w.n, 3)), w.id.copy(), w.type.copy())


def run_poiseuille_2d(kBT, seed):
    oracle = _setup()
    from paper_1807_09896_gb300 import inputs

    a, gamma, sigma, dt, mu_guess = POISEUILLE_2D[kBT]
    W, Lx, g, rho = 10.0, 30.0, 0.02, 4.0
    w = inputs.channel_2d(Lx, W, kBT=kBT, seed=seed)
    y = w.pos[:, 1].astype(np.float64)
    fl = w.type == 0
    w.vel[fl, 0] += (rho * g * y * (W - y) / (2 * mu_guess))[fl].astype(np.float32)
    p = oracle.Params(box=w.box, a_ff=a, a_fs=a, gamma=gamma, sigma=sigma, kBT=kBT, dt=dt,
                      g=(g, 0.0, 0.0), seed=seed)
    field = oracle.Field(w.phi, w.h)
    st = oracle.init_forces(_state(oracle, w), p)
    n_eq, n_block = int(300.0 / dt), int(100.0 / dt)
    for _ in range(n_eq):
        st = oracle.step(st, p, field)
    blocks = np.zeros((POISEUILLE_2D_BLOCKS, 100, 5))
    k = n_eq
    for b in range(POISEUILLE_2D_BLOCKS):
        for _ in range(n_block):
            st = oracle.step(st, p, field)
            k += 1
            if k % 10 == 0:
                oracle.profile(st.pos.astype(np.float32), st.vel, st.type, 1, 100, 0.0, W, out=blocks[b])
    return f"poiseuille2d_kBT{kBT:g}_seed{seed}", blocks


def run_cylinders(eps):
    oracle = _setup()
    from paper_1807_09896_gb300 import inputs

    L, mu, g, rho, kBT = 28.0, 3.41, 0.005, 4.0, 0.1
    r = L * math.sqrt(eps / math.pi)
    w = inputs.cylinder_2d(L, r, kBT=kBT, seed=1)
    fl = w.type == 0
    w.vel[fl, 0] += np.float32(eq20(eps) * rho * g * L * L / (4 * math.pi * mu))
    p = oracle.Params(box=w.box, a_ff=1.875, a_fs=1.875, gamma=45.0, sigma=3.0, kBT=kBT, dt=0.005,
                      g=(g, 0.0, 0.0), seed=0)
    field = oracle.Field(w.phi, w.h)
    st = oracle.init_forces(_state(oracle, w), p)
    for _ in range(100000):
        st = oracle.step(st, p, field)
    vs = np.zeros(40)
    for q in range(40):
        for _ in range(10000):
            st = oracle.step(st, p, field)
        vs[q] = st.vel[fl, 0].sum() / fl.sum()
    return f"cylinders_eps{eps:g}", vs


def run_channel_slice(kind):
    oracle = _setup()
    from paper_1807_09896_gb300 import inputs

    Lx, Ly, H, g = SLICE
    w = inputs.channel(Lx, Ly, H, seed=0)
    vel = w.vel4()
    seed = 0
    if kind == "parabola":
        fl = w.type == 0
        z = w.pos[:, 2].astype(np.float64)
        vel[fl, 0] += (g * z * (H - z) / (2 * SLICE_NU0))[fl].astype(np.float32)
        seed = 1
    p = oracle.Params(box=w.box, g=(g, 0.0, 0.0), seed=seed)
    field = oracle.Field(w.phi, w.h)
    st = oracle.init_forces(_state(oracle, w, vel), p)
    blocks = np.zeros((SLICE_BLOCKS, SLICE_NB, 5))
    k = 0
    for b in range(SLICE_BLOCKS):
        for _ in range(SLICE_BLOCK_STEPS):
            st = oracle.step(st, p, field)
            k += 1
            if k % SLICE_EVERY == 0:
                oracle.profile(st.pos.astype(np.float32), st.vel, st.type, 2, SLICE_NB, 0.0, H,
                               out=blocks[b])
    return f"channel_slice_{kind}", blocks


def _job(spec):
    os.environ["OMP_NUM_THREADS"] = str(spec[-1])
    t0 = time.time()
    kind, arg = spec[0], spec[1]
    if kind == "p2d":
        name, data = run_poiseuille_2d(*arg)
    elif kind == "cyl":
        name, data = run_cylinders(arg)
    else:
        name, data = run_channel_slice(arg)
    print(f"{name}: {time.time() - t0:.0f} s", flush=True)
    return name, data


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=4)
    ap.add_argument("--threads", type=int, default=2)
    ap.add_argument("--only", nargs="*", default=None)
    args = ap.parse_args()
    specs = [("p2d", (kBT, seed)) for kBT in POISEUILLE_2D for seed in POISEUILLE_2D_SEEDS]
    specs += [("cyl", eps) for eps in CYLINDER_EPS]
    specs += [("slice", kind) for kind in ("startup", "parabola")]
    if args.only:
        specs = [s for s in specs if any(o in f"{s[0]}{s[1]}" for o in args.only)]
    specs = [s + (args.threads,) for s in specs]
    old = dict(np.load(OUT)) if os.path.exists(OUT) else {}
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        for name, data in pool.imap_unordered(_job, specs):
            old[name] = data
            np.savez(OUT, **old)


if __name__ == "__main__":
    main()
