#!/usr/bin/env python
"""Throughput of the phase-field no-slip DPD time step on GB300 (particle-steps/s).

A "step" is one full time step of the path: drift + bounce-back reflection +
cell key (integrate), cell-count scan, counting sort into cell order, pair force
(conservative + dissipative + Philox random, Eqs. 3-10) + closing half-kick.

Default workload: a plane Poiseuille channel at the paper's DPD parameters
(rho = 3, a_ff = a_fs = 25, gamma = 4.5, sigma = 3, kBT = 1, dt = 0.01), fluid gap
64 r_c between phase-field walls, box 80 x 64 x 66 r_c, ~983k fluid + ~31k frozen
wall particles, body force g_x = 0.01.  Synthetic, seeded inputs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is device time of K steps replayed from
CUDA graphs with the state resident in HBM; `e2e` is the same metric through the
public C ABI from pinned host buffers (load state, K steps, read profile and
state back); `roofline` is the pair-force kernel's achieved ALU op rate against
the lane peak; `cpu_baseline` is the FP64 oracle on a bounded slice of the same
workload on this host's cores.  `--impl reference` times that oracle alone.
With N > 1 every rank runs its own independent replica (weak scaling; the path
has no exchange step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Phase-field relaxation (Eq. 15): every node's value is read once and its new value
# written once; the 18 neighbour reads are served by L1/L2.
PHASE_FIELD_BYTES_PER_NODE = 8
# Algorithmic work of the pair-force kernel, per fluid particle (the per-unit
# figures of the design notes): every candidate of the 27 surrounding cells costs
# ~13 simple ops (separation, minimum image, r^2, compare); every pair inside r_c
# costs ~115 (Philox4x32-10 ~70 integer ops, Box-Muller ~15, pair force ~30).
# At rho = 3 with unit cells there are 81 candidates and 4/3 pi rho = 12.57 pairs.
OPS_PER_CANDIDATE = 13
OPS_PER_PAIR = 115
# Algorithmic HBM bytes per particle and step of the whole step: integrate 100,
# scan 5, scatter 11, per-cell order 12, gather 100, force 80 (design notes).
BYTES_PER_PARTICLE_STEP = 308
# Algorithmic bytes of each phase's kernel(s), per fluid particle, per solid
# particle and per cell (minimal traffic: every array the kernel must read or write,
# once).  integrate: pos, vel, frc in; pos, vel, vt, key out (a resting solid
# particle: pos in, key out); after a half-shell force the 24 B of
# fixed-point sums replace frc and are cleared (+32 B).  scan: count read twice,
# start written, and written again into count as the scatter's slot cursor.  scatter:
# key in, perm out, each cell's cursor read and written.  cell_sort: perm in and out,
# start in, count zeroed.  gather: perm, then pos, vt, vel in and out.
# force_pairs: full shell pos, vt, vel in, frc and vel out; half shell pos, vt in and
# 24 B of fixed-point sums.  (A step launches no finish pass: the drift does its work.)
PHASE_BYTES = {
    "integrate": {False: (100, 20, 0), True: (132, 20, 0)},
    "scan": (0, 0, 16),
    "scatter": (8, 8, 8),
    "cell_sort": (8, 8, 12),
    "gather": (100, 100, 0),
    "force_pairs": {False: (80, 16, 0), True: (56, 32, 0)},
}
SM_COUNT_GB300 = 152
LANES_PER_SM = 128
FALLBACK_HBM_GBS = 6800.0
GRAPH_STEPS = 20
E2E_REPEATS = 3


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="channel_1m",
                    choices=["channel_1m", "channel_200k", "spheres_c3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip adjoint and precision lines")
    ap.add_argument("--force-variant", type=int, default=-1,
                    help="use this pair-force launch shape instead of tuning (e.g. to profile it)")
    ap.add_argument("--batched-steps", type=int, default=2000)
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the extra workload lines (channel_200k, spheres_c3)")
    ap.add_argument("--timed-ms", type=float, default=1500.0,
                    help="repeat the K-step replay until about this much device time is timed")
    return ap.parse_args()


WORKLOADS = {
    # name: (Lx, Ly, gap H, g_x)
    "channel_1m": (80.0, 64.0, 64.0, 0.01),
    "channel_200k": (64.0, 32.0, 32.0, 0.01),
}
# complex geometry: periodic cube of edge L with nspheres non-overlapping solid
# spheres of radius U(rmin, rmax), fluid in the pores, body force g_x
SPHERE_WORKLOADS = {
    "spheres_c3": (100.0, 40, 6.0, 12.0, 0.005),
}


def reduce_over_ranks(ms: float, units: float, device=None):
    """Whole-job timing across ranks: the slowest rank's time and the total work.
    Single process: returned unchanged."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, units
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def _workload(name, seed):
    from paper_1807_09896_gb300 import inputs

    if name in SPHERE_WORKLOADS:
        L, nsph, rmin, rmax, gx = SPHERE_WORKLOADS[name]
        return inputs.sphere_pack(L, nsph, rmin, rmax, seed=seed), gx
    Lx, Ly, H, gx = WORKLOADS[name]
    return inputs.channel(Lx, Ly, H, seed=seed), gx


def _describe(name, w, gx):
    if name in SPHERE_WORKLOADS:
        L, nsph, rmin, rmax, _ = SPHERE_WORKLOADS[name]
        return (f"{name}: periodic cube {L:g}^3 r_c, {nsph} solid spheres of radius U({rmin:g}, "
                f"{rmax:g}), rho 3, a 25, gamma 4.5, sigma 3, kBT 1, dt 0.01, g_x {gx}")
    return (f"{name}: plane Poiseuille channel, box {w.box[0]:g}x{w.box[1]:g}x{w.box[2]:g} r_c, "
            f"gap {w.gap:g}, rho 3, a 25, gamma 4.5, sigma 3, kBT 1, dt 0.01, g_x {gx}")


def prepare_graphs(s, graph_steps):
    """Capture the step graphs of both buffer parities before any timing (a graph
    of an even number of steps starts and ends in the same buffers; one single
    step between the two replays flips the parity).  Advances 2 (graph_steps + 1)
    steps and leaves the state in the buffers it started in."""
    for _ in range(2):
        s.step(graph_steps)
        s.step(1)


def time_replays(s, steps, stream, torch, dev, target_ms, min_repeats=5, max_repeats=2000,
                 barrier=lambda: None):
    """Device time of `steps` steps replayed from the prebuilt graphs, as the median
    over R repeats (CUDA events on the library's stream around each call), with R
    sized so that about target_ms of device time is timed.  Returns (median ms, R,
    list of ms)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    est = max(e0.elapsed_time(e1), 1e-3)
    reps = int(min(max_repeats, max(min_repeats, math.ceil(target_ms / est))))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    barrier()
    torch.cuda.synchronize(dev)
    for a, b in ev:
        a.record(stream)
        s.step(steps)
        b.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    times = [a.elapsed_time(b) for a, b in ev]
    return statistics.median(times), reps, times


def per_kernel_roofline(ph, newton3, n_fluid, n_solid, ncells, hbm_peak, hbm_src):
    """HBM fraction of each phase's kernel(s): algorithmic bytes per launch over the
    phase's mean CUDA-event time."""
    out = {}
    for name, ms in ph.items():
        if name not in PHASE_BYTES or ms <= 0.0:
            continue
        spec = PHASE_BYTES[name]
        if isinstance(spec, dict):
            spec = spec[newton3]
        bpf, bps, bpc = spec
        nbytes = bpf * n_fluid + bps * n_solid + bpc * ncells
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "bytes_per_launch": nbytes, "achieved": gbs, "peak": hbm_peak,
                     "unit": "GB/s", "frac": gbs / hbm_peak, "peak_source": hbm_src,
                     "bound": "alu" if name == "force_pairs" else "hbm"}
    return out


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            hbm = d.get("hbm_gbs") or d.get("hbm_GBs")
            return float(hbm), "measured", d
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback", {}


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.proc = None
        # raw samples go to DPD_CLOCKS_DIR if set, else the temporary directory; the
        # JSON line carries their summary
        out_dir = os.environ.get("DPD_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")
        self.uuid = device_uuid

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons, "samples": len(rows)}


def _source_hash():
    h = hashlib.sha256()
    for f in ("dpd_force.cu", "dpd_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1807_09896_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _force_traffic():
    """DRAM bytes per force launch from the committed ncu summary, if it still
    describes the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "force_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("source_hash") != _source_hash():
        return None
    return d


def cpu_oracle_rate(name, budget_s=10.0, min_steps=2, max_steps=None, warmup=0, seed=0):
    """FP64 oracle throughput on a slice of the workload (same gap and density,
    smaller Lx x Ly sized to the time budget): `warmup` untimed steps, then timed
    steps until the budget is used (at least min_steps, at most max_steps)."""
    import numpy as np

    import oracle
    from paper_1807_09896_gb300 import inputs

    if name in SPHERE_WORKLOADS:
        return _cpu_oracle_rate_whole(name, budget_s, min_steps, max_steps, warmup, seed)
    Lx, Ly, H, gx = WORKLOADS[name]
    # calibrate on a small slice, then size the slice to the budget
    probe = inputs.channel(6.0, 6.0, H, seed=seed)
    p = oracle.Params(box=probe.box, g=(gx, 0, 0), seed=seed)
    st = oracle.State(probe.pos.astype(np.float64), probe.vel.astype(np.float64),
                      np.zeros((probe.n, 3)), probe.id.copy(), probe.type.copy())
    st = oracle.init_forces(st, p)
    t0 = time.perf_counter()
    oracle.step(st, p, oracle.Field(probe.phi, probe.h))
    rate = probe.n_fluid / max(time.perf_counter() - t0, 1e-6)
    planned = max_steps if max_steps else max(min_steps, 3)
    per_step = budget_s / planned
    area = max(16.0, min(Lx * Ly, rate * per_step / (3.0 * H)))
    side_x = min(Lx, max(4.0, math.floor(math.sqrt(area * Lx / Ly))))
    side_y = min(Ly, max(4.0, math.floor(area / side_x)))
    w = inputs.channel(side_x, side_y, H, seed=seed)
    p = oracle.Params(box=w.box, g=(gx, 0, 0), seed=seed)
    field = oracle.Field(w.phi, w.h)
    st = oracle.State(w.pos.astype(np.float64), w.vel.astype(np.float64), np.zeros((w.n, 3)),
                      w.id.copy(), w.type.copy())
    st = oracle.init_forces(st, p)
    for _ in range(warmup):
        st = oracle.step(st, p, field)
    done, t0 = 0, time.perf_counter()
    while True:
        st = oracle.step(st, p, field)
        done += 1
        el = time.perf_counter() - t0
        if max_steps and done >= max_steps:
            break
        if not max_steps and done >= min_steps and el >= budget_s:
            break
    return {"value": w.n_fluid * done / el, "unit": "particle-steps/s",
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"channel slice {side_x:g}x{side_y:g} r_c, gap {H:g} ({w.n_fluid} fluid + "
                      f"{w.n_solid} solid particles) of the {Lx:g}x{Ly:g} workload, {done} FP64 "
                      f"steps in {el:.1f} s after {warmup} untimed"}


def _cpu_oracle_rate_whole(name, budget_s, min_steps, max_steps, warmup, seed):
    """FP64 oracle throughput on the whole workload (its steps take about a second)."""
    import numpy as np

    import oracle

    w, gx = _workload(name, seed)
    p = oracle.Params(box=w.box, g=(gx, 0, 0), seed=seed)
    field = oracle.Field(w.phi, w.h)
    st = oracle.State(w.pos.astype(np.float64), w.vel.astype(np.float64), np.zeros((w.n, 3)),
                      w.id.copy(), w.type.copy())
    st = oracle.init_forces(st, p)
    for _ in range(warmup):
        st = oracle.step(st, p, field)
    done, t0 = 0, time.perf_counter()
    while True:
        st = oracle.step(st, p, field)
        done += 1
        el = time.perf_counter() - t0
        if max_steps and done >= max_steps:
            break
        if not max_steps and done >= min_steps and el >= budget_s:
            break
    return {"value": w.n_fluid * done / el, "unit": "particle-steps/s",
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"the whole {name} workload ({w.n_fluid} fluid + {w.n_solid} solid "
                      f"particles), {done} FP64 steps in {el:.1f} s after {warmup} untimed"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # each timed step is one oracle step of a slice of the workload sized so that
    # the W + K steps take about two minutes
    budget = 120.0 * args.steps / max(1, args.steps + args.warmup)
    cb = cpu_oracle_rate(args.workload, budget_s=budget, max_steps=max(1, args.steps),
                         warmup=args.warmup)
    v = cb["value"]
    n_fluid = _workload(args.workload, 0)[0].n_fluid
    line = {
        "impl": "reference", "metric": "particle-steps/s", "value": v, "unit": "particle-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * n_fluid / v, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload,
                   "note": "FP64 CPU oracle on a slice of the workload; ms_per_step is the time one "
                           "step of the whole workload takes at the measured rate"},
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def measure_workload(dpd, torch, dev, stream, rank, name, steps, timed_ms, hbm_peak, hbm_src,
                     barrier):
    """Throughput line of another workload, measured like the headline one: tuned
    force shape, graphs captured first, median over repeats of a K-step replay."""
    t0 = time.perf_counter()
    w, gx = _workload(name, seed=rank)
    gen_s = time.perf_counter() - t0
    s = dpd.System.from_workload(w, g=(gx, 0.0, 0.0))
    dpd.dpd_set_stream(s.h, stream)
    s.set_option("use_graph", 1)
    s.set_option("graph_steps", GRAPH_STEPS)
    s.set_option("seed", rank)
    s.step(GRAPH_STEPS)
    chosen, _ = dpd.dpd_autotune(s.h, 3)
    newton3 = bool(s.get_option("force_newton3"))
    prepare_graphs(s, GRAPH_STEPS)
    ms, reps, _ = time_replays(s, steps, stream, torch, dev, timed_ms / 3, barrier=barrier)
    ms, units = reduce_over_ranks(ms, float(w.n_fluid) * steps, device=dev)
    ph = dpd.dpd_time_phases(s.h, min(steps, 20))
    st = s.stats()
    s.close()
    ncells = int(w.box[0]) * int(w.box[1]) * int(w.box[2])
    step_gbs = BYTES_PER_PARTICLE_STEP * (w.n_fluid + w.n_solid) * steps / (ms / 1e3) / 1e9
    return {"workload": _describe(name, w, gx), "n_fluid": w.n_fluid, "n_solid": w.n_solid,
            "value": units / (ms / 1e3), "unit": "particle-steps/s", "ms_per_step": ms / steps,
            "steps": steps, "repeats": reps, "force_launch_shape": chosen,
            "step_hbm": {"achieved": step_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": step_gbs / hbm_peak, "peak_source": hbm_src,
                         "bytes_per_particle_step": BYTES_PER_PARTICLE_STEP},
            "per_kernel": per_kernel_roofline(ph, newton3, w.n_fluid, w.n_solid, ncells, hbm_peak,
                                              hbm_src),
            "reflections": st[5], "fallbacks": st[6], "input_generation_s": gen_s}


def measure_batched(dpd, torch, dev, stream, rank, nsys=64, steps=200):
    """Ensemble of 64 uneven channels and sphere-pack pores (2k-60k fluid particles
    each): the batch (one launch per phase over all systems, graph replay) against
    the same systems stepped one after another, each with its own graphs."""
    from paper_1807_09896_gb300 import inputs

    ws = inputs.ensemble(nsys, seed=64 * rank)
    systems = []
    for k, w in enumerate(ws):
        gx = 0.01 if w.gap else 0.005
        s = dpd.System.from_workload(w, g=(gx, 0.0, 0.0), seed=k, system=k)
        dpd.dpd_set_stream(s.h, stream)
        systems.append(s)
    nf = sum(w.n_fluid for w in ws)
    b = dpd.Batch(systems, graph_steps=20)
    dpd.dpd_batch_set_stream(b.hb, stream)
    chosen, _ = dpd.dpd_batch_autotune(b.hb, 3)
    b.step(20)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_b = e0.elapsed_time(e1)
    for s in systems:
        s.set_option("use_graph", 1)
        s.set_option("graph_steps", 20)
        s.step(20)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for s in systems:
        s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_s = e0.elapsed_time(e1)
    b.close()
    for s in systems:
        s.close()
    return {"workload": f"{nsys} systems (alternating plane channels and sphere-pack pores, "
                        f"2k-60k fluid each, {nf} fluid in total)",
            "steps": steps, "value": nf * steps / (ms_b / 1e3), "unit": "particle-steps/s",
            "serial_value": nf * steps / (ms_s / 1e3), "speedup_vs_serial": ms_s / ms_b,
            "ms_per_step_batched": ms_b / steps, "ms_per_step_serial": ms_s / steps,
            "force_launch_shape": chosen}


def measure_adjoint(dpd, torch, dev, stream, nsteps=200, ckpt=20):
    """Adjoint window vs forward steps on the calibration channel 32 x 16 x 16
    (~25k fluid particles): the same 200 steps plain (graph replay) and with the
    near-wall loss gradient (forward + checkpointed recompute + reverse)."""
    from paper_1807_09896_gb300 import adjoint, inputs

    w = inputs.channel(32.0, 16.0, 16.0, seed=0)
    s = dpd.System.from_workload(w, g=(0.02, 0.0, 0.0))
    dpd.dpd_set_stream(s.h, stream)
    target = adjoint.poiseuille_wall_target(16.0, 0.02, 3.0, 0.9, 8, 0.25)
    loss = adjoint.NearWallLoss(0.0, 16.0, target)
    theta = (25.0, 4.5, 0.02)
    adjoint.window_loss_and_grad(s, theta, loss, nsteps, ckpt)  # warm-up
    s.step(nsteps)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    s.step(nsteps)
    torch.cuda.synchronize(dev)
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    L, g = adjoint.window_loss_and_grad(s, theta, loss, nsteps, ckpt)
    torch.cuda.synchronize(dev)
    t_adj = time.perf_counter() - t0
    s.close()
    return {"workload": f"channel 32x16x16 (gap 16), {w.n_fluid} fluid, {nsteps}-step window, "
                        f"checkpoint every {ckpt}",
            "forward_ms": 1e3 * t_fwd, "adjoint_ms": 1e3 * t_adj, "adjoint_over_forward": t_adj / t_fwd,
            "loss": L, "grad_a_fs_gamma_gx": [float(x) for x in g]}


def measure_phase_field(dpd, hbm_peak, hbm_src, iters=200):
    """Phase-field relaxation (Eq. 15) on the grid of the 1M-particle channel
    (320 x 256 x 264 nodes at h = 0.25, eps = 0.5) from a step function: one
    stencil launch per pseudo-time step, 4 B read + 4 B written per node."""
    import numpy as np

    nx, ny, nz, h = 320, 256, 264, 0.25
    z = (np.arange(nz) + 0.5) * h
    phi = np.broadcast_to(np.where((z > 1.0) & (z < 65.0), 1.0, -1.0)[:, None, None],
                          (nz, ny, nx)).astype(np.float32)
    dpd.dpd_relax_phase_field(phi, h, 0.5, 10, 0.04)  # warm-up
    _, ms = dpd.dpd_relax_phase_field(phi, h, 0.5, iters, 0.04)
    gbs = PHASE_FIELD_BYTES_PER_NODE * nx * ny * nz / (ms * 1e-3) / 1e9
    return {"kernel": "k_relax (Eq. 15, 19-point stencil)", "grid": [nx, ny, nz],
            "iters": iters, "ms_per_iter": ms, "bound": "hbm", "achieved": gbs,
            "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak, "peak_source": hbm_src,
            "bytes_per_node": PHASE_FIELD_BYTES_PER_NODE}


def measure_precision(dpd, nsteps=100):
    """Binary32 GPU against the binary64 oracle from identical state on the
    10 x 10 x 10-gap channel: one step (force, position, velocity errors) and the
    divergence of the two trajectories over nsteps steps."""
    import numpy as np

    import oracle
    from paper_1807_09896_gb300 import inputs

    w = inputs.channel(10.0, 10.0, 10.0, seed=0)
    p = oracle.Params(box=w.box, g=(0.02, 0.0, 0.0), seed=0)
    s = dpd.System.from_workload(w, g=(0.02, 0.0, 0.0))
    field = oracle.Field(w.phi, w.h)
    pos4, vel4, f4, ids, types = s.state()
    st = oracle.State(pos4[:, :3].astype(np.float64), vel4[:, :3].astype(np.float64),
                      f4[:, :3].astype(np.float64), ids, types, 0)
    fluid = types == 0
    s.step(1)
    g1 = s.state()
    o1 = oracle.step(st, p, field)
    scale = np.abs(o1.frc[fluid]).max()
    ferr = float(np.abs(g1[2][fluid, :3] - o1.frc[fluid]).max() / scale)
    L = np.asarray(w.box)
    dp = g1[0][:, :3] - o1.pos
    dp -= L * np.round(dp / L)
    perr = float(np.abs(dp).max())
    verr = float(np.abs(g1[1][fluid, :3] - o1.vel[fluid]).max())
    o = o1
    div = {}
    for k in range(2, nsteps + 1):
        s.step(1)
        o = oracle.step(o, p, field)
        if k in (10, 30, 100):
            g = s.state()
            d = g[0][:, :3] - o.pos
            d -= L * np.round(d / L)
            div[str(k)] = {"rms_position": float(np.sqrt((d[fluid] ** 2).sum(1).mean())),
                           "rms_velocity": float(np.sqrt(((g[1][fluid, :3] - o.vel[fluid]) ** 2).sum(1).mean()))}
    s.close()
    return {"workload": f"channel 10x10x10 gap, {w.n_fluid} fluid + {w.n_solid} solid",
            "one_step": {"force_max_err_over_max_force": ferr, "position_max_abs": perr,
                         "velocity_max_abs": verr},
            "trajectory_divergence": div,
            "note": "FP32 force/integrate, FP64 sums; trajectories of a chaotic system diverge"}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1807_09896_gb300 import _build, dpd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)  # before the process group, so NCCL binds this rank's GPU
    if world > 1:
        dist.init_process_group("nccl")
    _build.build()
    dev = torch.device("cuda", local)
    # a real stream (not the legacy default stream) so that the library can capture
    # CUDA graphs on it and the events below order with its work
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    w, gx = _workload(args.workload, seed=rank)
    s = dpd.System.from_workload(w, g=(gx, 0.0, 0.0))
    dpd.dpd_set_stream(s.h, stream)
    s.set_option("use_graph", 1)
    s.set_option("graph_steps", GRAPH_STEPS)
    s.set_option("seed", rank)

    def barrier():
        if world > 1:
            dist.barrier()

    s.step(args.warmup)
    # pick the pair-force launch shape on this device (tuning leaves the state as it was)
    if args.force_variant >= 0:
        s.set_option("force_variant", args.force_variant)
        chosen = args.force_variant
    else:
        chosen, _ = dpd.dpd_autotune(s.h, 5)
    newton3 = bool(s.get_option("force_newton3"))
    # the timed region replays graphs only: capture them first (tuning drops them)
    prepare_graphs(s, GRAPH_STEPS)
    torch.cuda.synchronize(dev)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.3)
    launches0 = s.get_option("kernel_launches")
    ms, reps, rep_ms = time_replays(s, args.steps, stream, torch, dev, args.timed_ms,
                                    barrier=barrier)
    ck = clocks.stop()
    # kernels of one timed K-step call (every repeat launches the same ones)
    launches = int(round((s.get_option("kernel_launches") - launches0) / (reps + 1)))
    ms, units = reduce_over_ranks(ms, float(w.n_fluid) * args.steps, device=dev)
    value = units / (ms / 1e3)

    # phase durations with CUDA events on the library's stream (same launches, no graph)
    nph = min(args.steps, 50)
    ph = dpd.dpd_time_phases(s.h, nph)
    force_ms = ph["force_pairs"]
    # the unit of work is fixed per particle-step (27 cells of candidates, every pair in
    # r_c), whichever algorithm runs; the half shell's own count is reported beside it
    cand = 27 * 3.0                    # 27 cells of unit volume at rho = 3
    pairs = 4.0 / 3.0 * math.pi * 3.0  # neighbours within r_c at rho = 3
    ops_unit = cand * OPS_PER_CANDIDATE + pairs * OPS_PER_PAIR
    ops_own = ops_unit / 2.0 if newton3 else ops_unit  # half shell: half the tests and pairs
    ops_per_launch = w.n_fluid * ops_unit
    achieved_tops = ops_per_launch / (force_ms / 1e3) / 1e12
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = (ck or {}).get("sm_max_mhz") or 2070.0
    peak_tops = sm_count * LANES_PER_SM * max_mhz * 1e6 / 1e12
    traffic = (_force_traffic() or {}).get("variants", {}).get(str(chosen))
    hbm_peak, hbm_src, _ = _peaks()
    step_gbs = BYTES_PER_PARTICLE_STEP * (w.n_fluid + w.n_solid) * args.steps / (ms / 1e3) / 1e9
    ncells = int(w.box[0]) * int(w.box[1]) * int(w.box[2])
    kernels = per_kernel_roofline(ph, newton3, w.n_fluid, w.n_solid, ncells, hbm_peak, hbm_src)

    # end to end through the public API from pinned host buffers
    pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    hp, hv = pin((w.n, 4), torch.float32), pin((w.n, 4), torch.float32)
    hi, ht = pin((w.n,), torch.int32), pin((w.n,), torch.uint8)
    hp[:], hv[:], hi[:], ht[:] = w.pos4(), w.vel4(), w.id, w.type
    op, ov, of = (pin((w.n, 4), torch.float32) for _ in range(3))
    oi, ot = pin((w.n,), torch.int32), pin((w.n,), torch.uint8)
    nb = 64
    prof = pin((nb, 5), torch.float64)
    prof_hi = w.gap if w.gap else w.box[2]
    e2e_times = []
    for _ in range(E2E_REPEATS):
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s.set_particles(hp, hv, hi, ht)
        s.step(args.steps)
        dpd.dpd_velocity_profile(s.h, 2, nb, 0.0, prof_hi, mode=1, out=prof)
        dpd.dpd_get_state(s.h, op, ov, of, oi, ot)
        torch.cuda.synchronize(dev)
        e2e_times.append(time.perf_counter() - t0)
    barrier()
    e2e_s = statistics.median(e2e_times)
    e2e_s, e2e_units = reduce_over_ranks(e2e_s, float(w.n_fluid) * args.steps, device=dev)
    e2e = e2e_units / e2e_s
    h2d = w.n * (16 + 16 + 4 + 1)
    d2h = w.n * (16 * 3 + 4 + 1) + nb * 5 * 8
    st = s.stats()
    s.close()

    extra = {}
    if not args.no_workloads:
        for name in ("channel_200k", "spheres_c3"):
            if name != args.workload:
                extra[name] = measure_workload(dpd, torch, dev, stream, rank, name, args.steps,
                                               args.timed_ms, hbm_peak, hbm_src, barrier)
    batched = None if args.no_batched else measure_batched(dpd, torch, dev, stream, rank,
                                                            steps=args.batched_steps)
    adj = None if args.no_extras else measure_adjoint(dpd, torch, dev, stream)
    precision = None if (args.no_extras or rank != 0) else measure_precision(dpd)
    phase_field = None if (args.no_extras or rank != 0) else measure_phase_field(dpd, hbm_peak, hbm_src)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(args.workload, budget_s=10.0)

    if rank == 0:
        line = {
            "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {
                "workload": _describe(args.workload, w, gx),
                "n_fluid": w.n_fluid, "n_solid": w.n_solid,
                "value_counts": "fluid particles only",
                "l2": "inputs larger than L2: particle state 2 x %.0f MB + phase field %.0f MB" % (
                    w.n * 64 / 1e6, w.phi.nbytes / 1e6),
                "graph_steps": GRAPH_STEPS, "parallelism": f"replicas x{world}",
                "force_launch_shape": chosen,
                "timing": f"median over {reps} repeats of the K-step call (graphs captured before "
                          f"timing; repeats {min(rep_ms):.4f}-{max(rep_ms):.4f} ms)",
            },
            "roofline": {
                "kernel": ("k_force_n3 (half-shell pair force, fixed-point sums; the next drift "
                           "converts them and completes the closing kick)" if newton3 else
                           "k_force (full-shell pair force + closing half-kick)"),
                "bound": "alu",
                "ops_per_particle": ops_unit, "ops_per_particle_own_algorithm": ops_own,
                "achieved": achieved_tops, "peak": peak_tops, "unit": "Tops/s",
                "frac": achieved_tops / peak_tops,
                "peak_source": f"{sm_count} SMs x {LANES_PER_SM} lanes x {max_mhz:g} MHz",
                "force_ms_per_launch": force_ms, "phase_ms": ph,
                "traffic": (traffic or {}).get("bytes_per_launch_full"),
                "step_hbm": {"achieved": step_gbs, "peak": hbm_peak, "unit": "GB/s",
                             "frac": step_gbs / hbm_peak, "peak_source": hbm_src,
                             "bytes_per_particle_step": BYTES_PER_PARTICLE_STEP},
                "per_kernel": kernels,
            },
            "e2e": {"value": e2e, "unit": "particle-steps/s",
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                    "note": f"pinned host state in, K steps, profile + state out, per call; median "
                            f"of {E2E_REPEATS} calls"},
            "gpu_launches": launches,
            "clocks": ck,
            "cpu_baseline": cpu,
            "diagnostics": {"reflections": st[5], "fallbacks": st[6]},
            "workloads": extra,
            "batched": batched,
            "adjoint": adj,
            "fp32_vs_fp64": precision,
            "phase_field_relaxation": phase_field,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
