"""Shared test infrastructure: building matching CUDA-path and oracle lattices
from the same parameters and comparing their outputs by velocity vector."""
import numpy as np

from oracle import oracle as O
from paper_2605_14505_gb300 import lbm

PAIR_NAMES = {0: "27x19", 1: "19x7"}


def gpu_sim(params, storage="fp32"):
    return lbm.Simulation(params, storage=storage)


def oracle_for(params):
    qf, qg = lbm.PAIR_Q[params.pair]
    op = O.lattice_params(params.nx, params.ny, params.nz, qf, qg, params.forcing, params.tau_f,
                          params.tau_g, params.G, params.beta, rho0=params.rho0,
                          scalar_mode=params.scalar_mode, sc_shift=params.sc_shift)
    return O.OracleSim(op)


def slot_map(q):
    """perm[i] = oracle index of the velocity in library slot i."""
    e_gpu, _, _ = lbm.lbm_velocity_set(q)
    e_orc, _, _ = O.stencil(q)
    lut = {tuple(v): j for j, v in enumerate(e_orc)}
    return np.array([lut[tuple(v)] for v in e_gpu])


def lattice_params(nx, ny, nz, pair, forcing, tau_f, tau_g, G, beta, rho0=1.0, scalar_mode=0,
                   sc_shift=1.0, U0=0.04):
    p = lbm.lbm_params()
    p.nx, p.ny, p.nz = nx, ny, nz
    p.pair = lbm.PAIRS[pair] if isinstance(pair, str) else pair
    p.forcing = lbm.FORCINGS[forcing] if isinstance(forcing, str) else forcing
    p.storage = 0
    p.scalar_mode = scalar_mode
    p.tau_f, p.tau_g, p.G, p.beta, p.rho0, p.sc_shift = tau_f, tau_g, G, beta, rho0, sc_shift
    p.U0 = U0
    p.L = nx / (2 * np.pi)
    return p


def rel_err(a, b, scale=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.max(np.abs(b)) if scale is None else scale
    return float(np.max(np.abs(a - b)) / s) if s > 0 else float(np.max(np.abs(a - b)))
