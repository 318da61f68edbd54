"""Checks of the closed-form channel flows the flow tests compare with (CPU only).

The start-up series must vanish at t = 0, reach the steady parabola (Eq. 18) at late
times, vanish at the effective walls, and satisfy u_t = nu u_zz + g; the fit must
recover known parameters from noisy model data; the jackknife error of a plain mean
must be the standard error.
"""
import numpy as np

from flow_analysis import (bin_average, channel_velocity, fit_channel, jackknife,
                           parabola_fit)

G, NU, H = 0.01, 0.3, 32.0


def test_startup_series_starts_at_rest_and_ends_at_the_parabola():
    z = np.linspace(0.3, H - 0.3, 41)
    assert np.abs(channel_velocity(z, [0.0], G, NU, H, 0.0, nmax=4001)).max() < 2e-5
    steady = G * z * (H - z) / (2 * NU)
    late = channel_velocity(z, [1e5], G, NU, H, 0.0)
    np.testing.assert_allclose(late, steady, rtol=1e-12, atol=1e-12)
    # Eq. 19: the mean of the parabola is 2/3 of its maximum
    zz = np.linspace(0, H, 200001)
    u = G * zz * (H - zz) / (2 * NU)
    assert abs(np.trapezoid(u, zz) / H / u.max() - 2.0 / 3.0) < 1e-9


def test_startup_series_vanishes_at_the_effective_walls():
    for b in (0.0, 0.2, -0.1):
        for t in (0.5, 10.0, 300.0):
            u = channel_velocity(np.array([-b, H + b]), [t], G, NU, H, b)
            assert np.abs(u).max() < 1e-12


def test_startup_series_solves_the_diffusion_equation_with_forcing():
    z = np.linspace(4.0, 28.0, 13)
    t, dt, dz = 40.0, 1e-3, 1e-3
    u_t = (channel_velocity(z, [t + dt], G, NU, H, 0.1) -
           channel_velocity(z, [t - dt], G, NU, H, 0.1)) / (2 * dt)
    u_zz = (channel_velocity(z + dz, [t], G, NU, H, 0.1) - 2 * channel_velocity(z, [t], G, NU, H, 0.1) +
            channel_velocity(z - dz, [t], G, NU, H, 0.1)) / dz ** 2
    np.testing.assert_allclose(u_t, NU * u_zz + G, atol=2e-6)


def test_relaxation_from_another_parabola():
    z = np.linspace(1.0, H - 1.0, 9)
    nu0 = 0.25
    u0 = channel_velocity(z, [0.0], G, NU, H, 0.0, nu0=nu0, nmax=4001)
    np.testing.assert_allclose(u0, G * z * (H - z) / (2 * nu0), rtol=1e-4)
    np.testing.assert_allclose(channel_velocity(z, [1e5], G, NU, H, 0.0, nu0=nu0),
                               G * z * (H - z) / (2 * NU), rtol=1e-12)


def test_bin_average_is_exact_for_polynomials():
    got = bin_average(lambda z: z ** 3, 0.0, 0.5, 4)
    edges = np.arange(5) * 0.5
    exact = (edges[1:] ** 4 - edges[:-1] ** 4) / 4 / 0.5
    np.testing.assert_allclose(got, exact, rtol=1e-13)


def test_fit_recovers_viscosity_and_slip_length_from_noisy_data():
    rng = np.random.default_rng(3)
    nbins, width, nblk = 64, 0.5, 6
    times = [0.1 * np.arange(100 * k + 1, 100 * (k + 1) + 1) for k in range(nblk)]
    true_nu, true_b = 0.29, 0.12
    u = np.array([bin_average(lambda z: channel_velocity(z, t, G, true_nu, H, true_b), 0.0,
                              width, nbins) for t in times])
    u += rng.normal(0, 0.003, size=u.shape)
    zc = (np.arange(nbins) + 0.5) * width
    mask = (zc > 1.0) & (zc < H - 1.0)

    def est(keep):
        return fit_channel(u[keep], [times[k] for k in keep], mask, G, H, 0.0, width)[0]

    (nu, b), (enu, eb) = jackknife(est, nblk)
    assert abs(nu - true_nu) < 4 * enu + 1e-4 and enu < 0.01
    assert abs(b - true_b) < 4 * eb + 1e-3 and eb < 0.05


def test_jackknife_of_a_mean_is_the_standard_error():
    x = np.random.default_rng(1).normal(size=12)
    m, e = jackknife(lambda keep: x[keep].mean(), len(x))
    assert abs(m - x.mean()) < 1e-15
    assert abs(e - x.std(ddof=1) / np.sqrt(len(x))) < 1e-12


def test_parabola_fit_finds_zeros_and_maximum():
    zc = np.linspace(0.25, 9.75, 20)
    u = 0.3 * (zc + 0.2) * (10.2 - zc)
    umax, (z0, z1), _ = parabola_fit(zc, u, np.ones(20, bool))
    assert abs(z0 + 0.2) < 1e-9 and abs(z1 - 10.2) < 1e-9
    assert abs(umax - 0.3 * 5.2 * 5.2) < 1e-9
