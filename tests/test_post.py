"""Host post-processing (Eqs. 24, 27-29, central-difference dissipation,
kinetic-energy spectrum) against closed forms."""
import numpy as np

import stgv_inputs as I
from paper_2605_14505_gb300 import post


def test_unit_conversion_and_total_energy():
    series = [{"step": s, "Ek": 2e-4, "Ep": 1e-5, "eps_k": 1e-8, "eps_p": 2e-9, "eps_k_curl": 9e-9}
              for s in (0, 100, 200)]
    U0, L = 0.04, 256 / (2 * np.pi)
    d = post.to_physical(series, U0, L)
    assert np.allclose(d["t"], np.array([0, 100, 200]) * U0 / L)
    assert np.allclose(d["Ek"], 2e-4 / U0 ** 2)
    assert np.allclose(d["eps_k"], 1e-8 * L / U0 ** 3)
    assert np.allclose(d["Etot"], d["Ek"] + d["Ep"])
    # records that carry their own paper-unit values are taken as they are
    phys = [dict(r, t=r["step"] * 1e-3, Ek_phys=1.0, Ep_phys=2.0, eps_k_phys=3.0, eps_p_phys=4.0,
                 eps_k_curl_phys=5.0) for r in series]
    d2 = post.to_physical(phys)
    assert np.allclose(d2["t"], [0.0, 0.1, 0.2]) and np.allclose(d2["Etot"], 3.0)
    assert np.allclose(d2["eps_p"], 4.0)


def test_central_difference_is_exact_on_quadratics():
    t = np.linspace(0, 3, 31)
    E = 1.0 - 0.2 * t + 0.05 * t ** 2
    assert np.allclose(post.total_dissipation_rate(t, E), 0.2 - 0.1 * t, atol=1e-12)


def test_buoyancy_reynolds_and_flux_coefficients():
    assert np.allclose(post.buoyancy_reynolds([0.01, 0.02], Re=1600, Fr=0.5), [4.0, 8.0])
    assert np.allclose(post.flux_coefficient([1.0, 3.0], [2.0, 4.0]), [0.5, 0.75])
    t = np.linspace(0, 40, 401)
    # constant rates: Gamma_b = ratio; Fr_t = eps / (N E) with N = 1/Fr
    assert abs(post.bulk_flux_coefficient(t, 0.3 * np.ones_like(t), np.ones_like(t)) - 0.3) < 1e-12
    assert abs(post.turbulent_froude(t, 0.2 * np.ones_like(t), 0.5 * np.ones_like(t), Fr=0.25) - 0.1) < 1e-12
    # the integrals stop at t = 30
    eps_p = np.where(t <= 30, 1.0, 100.0)
    assert abs(post.bulk_flux_coefficient(t, eps_p, np.ones_like(t)) - 1.0) < 1e-12


def test_spectrum_of_the_taylor_green_field():
    """Eq. 20 has all its energy in the |k| = sqrt(3) shell (rounded to 2),
    and the spectrum sums to <|u|^2>/2 (Parseval)."""
    n = 16
    _, u, _ = I.tgv_fields(n, 1.0)
    k, E = post.energy_spectrum(u, n)
    assert abs(E.sum() - 0.5 * np.mean(np.sum(u ** 2, axis=0))) < 1e-12
    assert abs(E[2] - 0.125) < 1e-12 and abs(E.sum() - E[2]) < 1e-12


def test_spectral_slope_and_peaks():
    k = np.arange(1, 40, dtype=float)
    assert abs(post.spectral_slope(k, 3.0 * k ** (-5.0 / 3.0), 4, 20) + 5.0 / 3.0) < 1e-12
    t = np.linspace(0, 20, 401)
    y = np.exp(-((t - 11.5) / 1.0) ** 2) + 0.8 * np.exp(-((t - 16.5) / 1.0) ** 2) + 0.3 * np.exp(-((t - 3) / 0.5) ** 2)
    p = post.peaks(t, y, 2)
    assert [round(a, 2) for a, _ in p] == [11.5, 16.5]
    # a wiggle on the main peak is not a second peak when a separation is asked for
    y2 = y + 0.02 * np.sin(40 * t) * np.exp(-((t - 11.5) / 1.0) ** 2)
    p2 = post.peaks(t, y2, 2, separation=2.0)
    assert abs(p2[0][0] - 11.5) < 0.3 and abs(p2[1][0] - 16.5) < 0.3


def test_energy_balance_and_pressure_field():
    t = np.linspace(0, 4, 81)
    eps = 0.01 * np.exp(-0.3 * t)
    Ek = 0.125 - 0.01 / 0.3 * (1 - np.exp(-0.3 * t))   # dE/dt = -eps exactly
    assert abs(post.energy_balance(t, Ek, eps, 0.5, 3.0)) < 1e-4
    rho = post.tgv_pressure_density(8, 0.04)
    # mean of (cos 2x + cos 2y)(cos 2z + 2) over the grid is 0: mass unchanged
    assert abs(rho.mean() - 1.0) < 1e-15 and rho.max() > 1.0
