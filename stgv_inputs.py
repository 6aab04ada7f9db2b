"""Seeded synthetic inputs for the stratified Taylor-Green vortex workloads.

This module is the one place both the CUDA path and the CPU oracle take their
inputs from. It holds none of the lattice Boltzmann arithmetic: it only lays
out initial macroscopic fields (the benchmark's Eq. 20 and a few textbook
single-mode fields) and draws uniform random numbers.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw c of stream `seed` is the finaliser applied to
seed + (c + 1) * 0x9E3779B97F4A7C15 (mod 2^64), i.e. the c-th output of the
sequence started at state `seed`. The CUDA library's on-device TGV
initialiser implements the same published definition independently.

All arrays are flat float64 with node index x + nx*(y + ny*z) (x fastest).
Node i sits at x_i = i * 2*pi/n (vertex-centred grid on the periodic box
[0, 2*pi)^3 of Section 2.4).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Outputs number `counters` (0-based) of the SplitMix64 stream started at `seed`."""
    with np.errstate(over="ignore"):
        c = np.asarray(counters, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, counters: np.ndarray) -> np.ndarray:
    """Uniform draws in [-1, 1): 2 * (top 53 bits / 2^53) - 1."""
    z = splitmix64(seed, counters)
    u01 = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u01 - 1.0


def grid_axes(nx: int, ny: int | None = None, nz: int | None = None):
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    x = np.arange(nx) * (2.0 * np.pi / nx)
    y = np.arange(ny) * (2.0 * np.pi / ny)
    z = np.arange(nz) * (2.0 * np.pi / nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def tgv_fields(n: int, U0: float, seed: int | None = None, noise_amp: float = 0.0):
    """Eq. 20 on an n^3 grid: u = U0 (sin x cos y cos z, -cos x sin y cos z, 0),
    rho = 1, rho' = 0. With a seed and noise_amp > 0, each velocity component a
    gets + noise_amp * U0 * xi, xi = uniform_pm1(seed, a*n^3 + node)."""
    X, Y, Z = grid_axes(n)
    n3 = n ** 3
    u = np.empty((3, n3))
    u[0] = U0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    u[1] = -U0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    u[2] = 0.0
    if seed is not None and noise_amp != 0.0:
        xi = uniform_pm1(seed, np.arange(3 * n3, dtype=np.uint64)).reshape(3, n3)
        u += noise_amp * U0 * xi
    return np.ones(n3), u, np.zeros(n3)


def neq_noise(n3: int, seed: int) -> np.ndarray:
    """(27, n3) uniform [-1, 1) draws indexed by the canonical velocity code
    (ex+1)*9 + (ey+1)*3 + (ez+1); used as a seeded non-equilibrium perturbation."""
    return uniform_pm1(seed, np.arange(27 * n3, dtype=np.uint64)).reshape(27, n3)


def random_fields(nx: int, ny: int, nz: int, seed: int, u_amp: float, rho_amp: float,
                  rho_p_amp: float):
    """Smooth-free random macroscopic fields: rho = 1 + rho_amp*xi, u = u_amp*xi,
    rho' = rho_p_amp*xi (independent draws), for one-step parity checks."""
    n3 = nx * ny * nz
    xi = uniform_pm1(seed, np.arange(5 * n3, dtype=np.uint64)).reshape(5, n3)
    return 1.0 + rho_amp * xi[0], u_amp * xi[1:4], rho_p_amp * xi[4]


def shear_wave_fields(n: int, amp: float, mode: int = 1):
    """u_x = amp * sin(mode * z), rho = 1, rho' = 0 (a single transverse shear mode)."""
    X, Y, Z = grid_axes(n)
    u = np.zeros((3, n ** 3))
    u[0] = amp * np.sin(mode * Z)
    return np.ones(n ** 3), u, np.zeros(n ** 3)


def density_mode_fields(n: int, amp: float, kx: int = 1, ky: int = 0, kz: int = 1):
    """u = 0, rho = 1, rho' = amp * cos(kx x + ky y + kz z): the initial state of a
    standing internal gravity wave."""
    X, Y, Z = grid_axes(n)
    return np.ones(n ** 3), np.zeros((3, n ** 3)), amp * np.cos(kx * X + ky * Y + kz * Z)
