"""Post-processing of the diagnostics time series (paper Sections 3.3-3.5).

These are host-side reductions of a few numbers per sample, not part of the
GPU update. The paper's units have U = L = 1: time t = step * U0 / L_LB,
energies / U0^2, dissipation rates * L_LB / U0^3, where L_LB = n / (2 pi);
the library's diagnostics records already carry those values.
"""
from __future__ import annotations

import numpy as np

_trapezoid = getattr(np, "trapezoid", None) or np.trapz


def to_physical(series, U0: float | None = None, L: float | None = None) -> dict:
    """Arrays of a diagnostics time series in the paper's units.

    Records from the library carry the paper-unit values themselves (lbm_diag:
    t, Ek_phys, ..., computed in the C library from the handle's U0 and L);
    those are used as they are. Records without them (or with NaN there, for
    lattice parameters made without U0 and L) are converted from the lattice
    values with the given U0 and L."""
    def have(d):
        return "t" in d and np.isfinite(d["t"])

    if all(have(d) for d in series):
        out = {"t": np.array([d["t"] for d in series], dtype=np.float64)}
        for key in ("Ek", "Ep", "eps_k", "eps_p", "eps_k_curl"):
            out[key] = np.array([d[key + "_phys"] for d in series], dtype=np.float64)
    else:
        if U0 is None or L is None:
            raise ValueError("records without paper-unit values need U0 and L")
        step = np.array([d["step"] for d in series], dtype=np.float64)
        out = {"t": step * U0 / L}
        for key in ("Ek", "Ep"):
            out[key] = np.array([d[key] for d in series]) / U0 ** 2
        for key in ("eps_k", "eps_p", "eps_k_curl"):
            out[key] = np.array([d[key] for d in series]) * L / U0 ** 3
    out["Etot"] = out["Ek"] + out["Ep"]          # Eq. 24
    return out


def total_dissipation_rate(t, Etot):
    """-dE_tot/dt by second-order central differences on a uniform time grid
    (one-sided second-order differences at the two ends), Sections 3.1, 3.3."""
    t = np.asarray(t, dtype=np.float64)
    E = np.asarray(Etot, dtype=np.float64)
    if len(t) < 3:
        raise ValueError("need at least three samples")
    return -np.gradient(E, t, edge_order=2)


def buoyancy_reynolds(eps_k, Re: float, Fr: float):
    """Eq. 27, R = eps_k / (nu N^2), with nu = 1/Re and N = 1/Fr (U = L = 1)."""
    return np.asarray(eps_k, dtype=np.float64) * Re * Fr ** 2


def flux_coefficient(eps_p, eps_k):
    """Gamma = eps_p / eps_k (Section 3.5)."""
    return np.asarray(eps_p, dtype=np.float64) / np.asarray(eps_k, dtype=np.float64)


def _integral(t, y, t_end):
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m = t <= t_end + 1e-12
    return _trapezoid(y[m], t[m])


def bulk_flux_coefficient(t, eps_p, eps_k, t_end: float = 30.0):
    """Eq. 28: Gamma_b = int_0^T eps_p dt / int_0^T eps_k dt (trapezoidal rule)."""
    return _integral(t, eps_p, t_end) / _integral(t, eps_k, t_end)


def turbulent_froude(t, eps_k, Ek, Fr: float, t_end: float = 30.0):
    """Eq. 29: Fr_t = int_0^T eps_k dt / (N int_0^T E_k dt), N = 1/Fr."""
    return _integral(t, eps_k, t_end) / ((1.0 / Fr) * _integral(t, Ek, t_end))


def energy_spectrum(u, n: int):
    """Shell-averaged kinetic-energy spectrum E(k) of a periodic velocity field
    u (3 x n^3, x fastest, any units) on [0, 2 pi)^3 (Section 3.5): the energy
    of all Fourier modes with round(|k|) = k, normalised so that
    sum_k E(k) = <|u|^2> / 2. Returns (k, E)."""
    u = np.asarray(u, dtype=np.float64).reshape(3, n, n, n)
    uh = np.fft.fftn(u, axes=(1, 2, 3)) / n ** 3
    e = 0.5 * np.sum(np.abs(uh) ** 2, axis=0)
    kk = np.fft.fftfreq(n, d=1.0 / n)
    KZ, KY, KX = np.meshgrid(kk, kk, kk, indexing="ij")
    shell = np.rint(np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)).astype(np.int64)
    E = np.bincount(shell.ravel(), weights=e.ravel())
    return np.arange(len(E)), E


def energy_spectrum_device(u, n: int):
    """energy_spectrum on the GPU: u is a CUDA tensor (3, n^3), x fastest. The
    3-D FFT is cuFFT through torch.fft (a library transform off the update
    path); the shells are summed with one bincount. Returns numpy (k, E)."""
    import torch

    uh = torch.fft.fftn(u.reshape(3, n, n, n), dim=(1, 2, 3)) / n ** 3
    e = 0.5 * (uh.real ** 2 + uh.imag ** 2).sum(dim=0)
    kk = torch.fft.fftfreq(n, d=1.0 / n, device=u.device, dtype=torch.float64)
    KZ, KY, KX = torch.meshgrid(kk, kk, kk, indexing="ij")
    shell = torch.round(torch.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)).to(torch.int64)
    E = torch.bincount(shell.flatten(), weights=e.flatten())
    E = E.cpu().numpy()
    return np.arange(len(E)), E


def spectral_slope(k, E, kmin: float, kmax: float) -> float:
    """Least-squares slope of log E against log k over kmin <= k <= kmax
    (the paper compares the inertial range with k^(-5/3), Section 3.5)."""
    k = np.asarray(k, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    m = (k >= kmin) & (k <= kmax) & (E > 0)
    return float(np.polyfit(np.log(k[m]), np.log(E[m]), 1)[0])


def peaks(t, y, count: int = 2, separation: float = 0.0):
    """The `count` highest interior local maxima of a sampled series at least
    `separation` apart in t (highest first, then the next highest outside the
    chosen ones' windows), as (t, y) pairs in time order."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    idx = [i for i in range(1, len(y) - 1) if y[i] > y[i - 1] and y[i] >= y[i + 1]]
    chosen = []
    for i in sorted(idx, key=lambda i: -y[i]):
        if all(abs(t[i] - t[j]) >= separation for j in chosen):
            chosen.append(i)
        if len(chosen) == count:
            break
    return [(float(t[i]), float(y[i])) for i in sorted(chosen)]


def energy_balance(t, Ek, eps, t0: float, t1: float) -> float:
    """Relative mismatch of the kinetic-energy budget over [t0, t1]:
    (E_k(t0) - E_k(t1)) / int_t0^t1 eps dt - 1, i.e. the window average of
    -dE_k/dt against that of eps (trapezoidal rule on the samples)."""
    t = np.asarray(t, dtype=np.float64)
    m = (t >= t0 - 1e-12) & (t <= t1 + 1e-12)
    tw, ew = t[m], np.asarray(eps, dtype=np.float64)[m]
    kw = np.asarray(Ek, dtype=np.float64)[m]
    return float((kw[0] - kw[-1]) / _trapezoid(ew, tw) - 1.0)


def tgv_pressure_density(n: int, U0: float, cs2: float = 1.0 / 3.0):
    """rho = 1 + p / cs^2 with the Taylor-Green pressure
    p = (U0^2 / 16) (cos 2x + cos 2y) (cos 2z + 2) on the vertex grid (the
    standard form of the initial pressure that Eq. 21 prints garbled), in
    lattice units, flat x fastest."""
    x = np.arange(n) * (2.0 * np.pi / n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    p = (U0 ** 2 / 16.0) * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    return (1.0 + p / cs2).ravel()
