"""The plain channel at its full size and length: a 64 x 32 r_c periodic channel with a
fluid gap of 32 r_c between phase-field walls (~197 k fluid + ~12 k wall particles,
rho 3, a 25, gamma 4.5, sigma 3, kBT 1, dt 0.01, g_x 0.01), 10^4 steps, velocity,
density and temperature in 64 bins across the gap (Sec. III.A, Eqs. 18-19).

The flow takes ~H^2 / nu ~ 3500 time units to become the steady parabola, and 10^4
steps are 100, so the profile is compared with the closed-form start-up solution
(Fourier series of the parabola relaxing under u_t = nu u_zz + g, test helper
flow_analysis) with the kinematic viscosity nu and a slip length b as the two fitted
parameters: b = 0 puts the no-slip planes exactly at the phi = 0 walls.  Ten blocks
of 1000 steps, sampled every 10 steps, give jackknife error bars.  A second run
starts from the steady parabola of the fitted viscosity and checks Eq. 19 (mean
velocity = 2/3 of the maximum) and the zeros of the fitted parabola.  Bins within
1 r_c of a wall are left out of every fit (the density is layered there, Sec. III.A).
The absolute viscosity is not pinned by the paper (it prints 2-D values only).
"""
import numpy as np
import pytest

from flow_analysis import bin_average, channel_velocity, fit_channel, jackknife, parabola_fit, profile_fields
from paper_1807_09896_gb300 import inputs
from parity_helpers import make_system, params_for

pytestmark = pytest.mark.gpu

LX, LY, H, G = 64.0, 32.0, 32.0, 0.01
NB, WIDTH = 64, 0.5
BLOCKS, BLOCK_STEPS, EVERY, DT = 10, 1000, 10, 0.01
ZC = (np.arange(NB) + 0.5) * WIDTH
INNER = (ZC > 1.0) & (ZC < H - 1.0)


def _run_blocks(w, seed, vel=None):
    p = params_for(w, g=(G, 0.0, 0.0), seed=seed)
    s = make_system(w, p, load=False)
    s.set_particles(w.pos4(), w.vel4() if vel is None else vel, w.id, w.type)
    samples = BLOCK_STEPS // EVERY
    profs, times = [], []
    s.set_option("sample_every", EVERY)
    for k in range(BLOCKS):
        s.profile(2, NB, 0.0, H, mode=3)
        s.step(BLOCK_STEPS)
        profs.append(s.profile(2, NB, 0.0, H, mode=2).copy())
        times.append(DT * EVERY * np.arange(k * samples + 1, (k + 1) * samples + 1))
    s.close()
    return np.array(profs), times, samples


@pytest.fixture(scope="module")
def startup():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_09896_gb300 import _build

    _build.build()
    w = inputs.channel(LX, LY, H, seed=0)
    profs, times, samples = _run_blocks(w, seed=0)
    u = np.array([profile_fields(pr, samples, LX * LY, WIDTH)[1] for pr in profs])

    def est(keep):
        return fit_channel(u[keep], [times[k] for k in keep], INNER, G, H, 0.0, WIDTH)[0]

    (nu, b), (enu, eb) = jackknife(est, BLOCKS)
    _, res = fit_channel(u, times, INNER, G, H, 0.0, WIDTH)
    return {"w": w, "profs": profs, "times": times, "samples": samples, "u": u, "nu": nu, "b": b,
            "enu": enu, "eb": eb, "res": res}


def test_startup_profile_follows_the_no_slip_series(startup):
    r = startup
    print(f"C2 start-up: nu = {r['nu']:.4f} +- {r['enu']:.4f}, slip length b = {r['b']:.4f} +- "
          f"{r['eb']:.4f} r_c, rms residual {np.sqrt((r['res'] ** 2).mean()):.4f}")
    assert r["eb"] < 0.05 and r["enu"] < 0.01
    # no slip at the phi = 0 walls: the effective wall is within 0.25 r_c (0.8% of the gap)
    assert abs(r["b"]) < 0.25
    # the 3-D rho = 3, a = 25 DPD fluid (parity unpinned; commonly quoted ~0.28-0.29)
    assert 0.24 < r["nu"] < 0.34
    # the series describes every block: residuals at the level of the thermal noise
    assert np.sqrt((r["res"] ** 2).mean()) < 0.01
    # the last block's centre velocity agrees with the model
    t = r["times"][-1]
    centre = INNER & (np.abs(ZC - H / 2) < 2)
    model = bin_average(lambda z: channel_velocity(z, t, G, r["nu"], H, r["b"]), 0.0, WIDTH, NB)
    assert np.abs(r["u"][-1][centre] - model[centre]).max() < 0.02


def test_density_and_temperature_are_flat_away_from_the_walls(startup):
    r = startup
    # per block (the mean flow grows over the run: pooled over all blocks its growth
    # would count as thermal motion), then averaged over the blocks
    fields = [profile_fields(pr, r["samples"], LX * LY, WIDTH, rho_ref=3.0) for pr in r["profs"]]
    dens = np.mean([f[0] for f in fields], axis=0)
    temp = np.mean([f[2] for f in fields], axis=0)
    prof = r["profs"].sum(axis=0)
    print(f"C2 density {dens[INNER].min():.4f}..{dens[INNER].max():.4f}, temperature "
          f"{temp[INNER].min():.4f}..{temp[INNER].max():.4f} (interior bins)")
    assert np.abs(dens[INNER] - 1.0).max() < 0.03
    assert np.abs(temp[INNER] - 1.0).max() < 0.03
    # nothing inside the solid: the bins span the fluid gap only, and they hold every
    # fluid particle of every sample
    assert abs(prof[:, 0].sum() / (r["samples"] * BLOCKS) - r["w"].n_fluid) < 0.5


def test_flow_from_the_fitted_parabola_keeps_eq_19(startup):
    r = startup
    w = r["w"]
    nu0 = r["nu"]
    vel = w.vel4()
    fl = w.type == 0
    z = w.pos[:, 2].astype(np.float64)
    vel[fl, 0] += (G * z * (H - z) / (2 * nu0))[fl].astype(np.float32)
    profs, times, samples = _run_blocks(w, seed=1, vel=vel)
    u = np.array([profile_fields(pr, samples, LX * LY, WIDTH)[1] for pr in profs])

    def est(keep):
        uk = u[keep].mean(axis=0)
        umax, (z0, z1), _ = parabola_fit(ZC, uk, INNER)
        cnt = profs[keep][:, :, 0].sum()
        ubar = profs[keep][:, :, 1].sum() / cnt
        return [ubar / umax, -z0, z1 - H, 3.0 * G * (H / 2) ** 2 / (2 * umax)]

    (ratio, b_lo, b_hi, mu), (er, eblo, ebhi, emu) = jackknife(est, BLOCKS)
    print(f"C2 from the parabola: vbar/vmax = {ratio:.4f} +- {er:.4f} (Eq. 19: 2/3), zeros "
          f"{b_lo:.3f} +- {eblo:.3f} and {b_hi:.3f} +- {ebhi:.3f} r_c beyond the walls, mu(vmax) "
          f"= {mu:.4f} +- {emu:.4f} (rho nu of the start-up fit: {3.0 * nu0:.4f})")
    assert abs(ratio - 2.0 / 3.0) < max(4 * er, 0.01)
    assert abs(b_lo) < 0.3 and abs(b_hi) < 0.3
    assert abs(mu / (3.0 * nu0) - 1.0) < 0.05


def _slice_blocks(kind):
    from golden.make_fp64_observables import SLICE, SLICE_NU0

    Lx, Ly, H_, g = SLICE
    w = inputs.channel(Lx, Ly, H_, seed=0)
    vel, seed = None, 0
    if kind == "parabola":
        vel = w.vel4()
        fl = w.type == 0
        z = w.pos[:, 2].astype(np.float64)
        vel[fl, 0] += (g * z * (H_ - z) / (2 * SLICE_NU0))[fl].astype(np.float32)
        seed = 1
    profs, times, samples = _run_blocks(w, seed=seed, vel=vel)
    return profs, times, samples, Lx * Ly


def _slice_observables(profs, times, samples, area, kind):
    from golden.make_fp64_observables import SLICE_NU0

    u = np.array([profile_fields(pr, samples, area, WIDTH)[1] for pr in profs])
    nu0 = SLICE_NU0 if kind == "parabola" else None
    return jackknife(lambda keep: fit_channel(u[keep], [times[k] for k in keep], INNER, G, H, 0.0,
                                              WIDTH, nu0=nu0)[0], BLOCKS)


@pytest.mark.parametrize("kind", ["startup", "parabola"])
def test_fp32_and_fp64_slices_agree_within_errors(startup, kind):
    """FP32 against FP64 for the fitted viscosity and slip length: a 16 x 8 slice of the
    same channel run on the GPU and by the binary64 oracle from the same start, seed and
    schedule (tests/golden/make_fp64_observables.py).  The trajectories separate, so the
    fits must agree within their combined jackknife errors."""
    import os

    fp64 = np.load(os.path.join(os.path.dirname(__file__), "golden", "fp64_observables.npz"))
    profs, times, samples, area = _slice_blocks(kind)
    (nu, b), (enu, eb) = _slice_observables(profs, times, samples, area, kind)
    (nu64, b64), (enu64, eb64) = _slice_observables(fp64[f"channel_slice_{kind}"], times, samples,
                                                    area, kind)
    print(f"C2 slice {kind}: nu binary32 {nu:.4f} +- {enu:.4f} binary64 {nu64:.4f} +- {enu64:.4f}; "
          f"b binary32 {b:.4f} +- {eb:.4f} binary64 {b64:.4f} +- {eb64:.4f} r_c")
    assert abs(nu - nu64) <= 4 * np.hypot(enu, enu64)
    assert abs(b - b64) <= 4 * np.hypot(eb, eb64)
