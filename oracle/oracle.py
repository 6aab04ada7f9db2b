"""Python view of the FP64 CPU oracle in ``oracle/stgv_oracle.c``.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``. Nothing in
the ``paper_2605_14505_gb300`` package imports this module, and this module
imports nothing from that package.

The oracle follows the paper's Section 2 (Eqs. 5-18, Table A.1) step by step
in FP64 with two-lattice pull streaming; see the header of stgv_oracle.c for
the readings it takes where the paper is silent or inconsistent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stgv_oracle.c")
_LIB = os.path.join(_HERE, "libstgv_oracle.so")

FORCING = {"guo": 0, "sc": 1, "edm": 2, "hcz": 3}
DIAG_NAMES = (
    "Ek", "Ep", "eps_k", "eps_p", "eps_k_curl",
    "mass_f", "mass_g", "mom_x", "mom_y", "mom_z", "umax",
)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE FP64: no fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = [
            "gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
            "-ffp-contract=off", "-o", _LIB + ".tmp", _SRC, "-lm",
        ]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("qf", ctypes.c_int), ("qg", ctypes.c_int),
        ("forcing", ctypes.c_int), ("scalar_mode", ctypes.c_int),
        ("tau_f", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("G", ctypes.c_double), ("beta", ctypes.c_double),
        ("rho0", ctypes.c_double), ("sc_shift", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.orc_stencil_info.argtypes = [ctypes.c_int, ip, dp, dp]
            L.orc_equilibrium.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [dp]
            L.orc_params_from_physics.argtypes = [
                ctypes.POINTER(OrcParams), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ]
            L.orc_create.argtypes = [ctypes.POINTER(OrcParams)]
            L.orc_create.restype = ctypes.c_void_p
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_step_count.argtypes = [ctypes.c_void_p]
            L.orc_step_count.restype = ctypes.c_longlong
            L.orc_init_fields.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp, ctypes.c_double]
            L.orc_set_populations.argtypes = [ctypes.c_void_p, dp, dp]
            L.orc_get_populations.argtypes = [ctypes.c_void_p, dp, dp]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_longlong]
            L.orc_get_fields.argtypes = [ctypes.c_void_p, dp, dp, dp]
            L.orc_diagnostics.argtypes = [ctypes.c_void_p, dp]
            if L.orc_sizeof_params() != ctypes.sizeof(OrcParams):
                raise RuntimeError("oracle parameter struct layout mismatch")
            _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def stencil(q: int):
    """Velocity set of Table A.1 as generated by the oracle: (e[q,3], w[q], cs2)."""
    e = np.zeros(27 * 3, dtype=np.int32)
    w = np.zeros(27, dtype=np.float64)
    cs2 = ctypes.c_double()
    n = lib().orc_stencil_info(q, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                               ctypes.byref(cs2))
    if n < 0:
        raise ValueError(f"unknown stencil Q{q}")
    return e[: 3 * n].reshape(n, 3).copy(), w[:n].copy(), cs2.value


def equilibrium(q: int, rho: float, u) -> np.ndarray:
    """Eq. 9 for one node."""
    out = np.zeros(27, dtype=np.float64)
    n = lib().orc_equilibrium(q, rho, float(u[0]), float(u[1]), float(u[2]), _dp(out))
    if n < 0:
        raise ValueError(f"unknown stencil Q{q}")
    return out[:n].copy()


def params_from_physics(n, qf, qg, forcing, Re, Fr, Sc, U0) -> OrcParams:
    p = OrcParams()
    if isinstance(forcing, str):
        forcing = FORCING[forcing]
    rc = lib().orc_params_from_physics(ctypes.byref(p), n, qf, qg, forcing, Re, Fr, Sc, U0)
    if rc != 0:
        raise ValueError("invalid physical parameters")
    return p


def lattice_params(nx, ny, nz, qf, qg, forcing, tau_f, tau_g, G, beta, rho0=1.0,
                   scalar_mode=0, sc_shift=1.0) -> OrcParams:
    if isinstance(forcing, str):
        forcing = FORCING[forcing]
    return OrcParams(nx, ny, nz, qf, qg, forcing, scalar_mode, tau_f, tau_g, G, beta, rho0,
                     sc_shift)


class OracleSim:
    """One oracle lattice. Arrays are flat FP64, node index x + nx*(y + ny*z)."""

    def __init__(self, params: OrcParams):
        self.params = params
        self._h = lib().orc_create(ctypes.byref(params))
        if not self._h:
            raise ValueError("oracle rejected parameters")
        self.nx, self.ny, self.nz = params.nx, params.ny, params.nz
        self.n3 = self.nx * self.ny * self.nz
        self.ef, self.wf, self.cs2f = stencil(params.qf)
        self.eg, self.wg, self.cs2g = stencil(params.qg)

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def step_count(self) -> int:
        return int(lib().orc_step_count(self._h))

    def init_fields(self, rho, u, rho_p, xi_f=None, xi_g=None, amp=0.0):
        rho, u, rho_p = _f64(rho), _f64(u), _f64(rho_p)
        assert rho.size == self.n3 and u.size == 3 * self.n3 and rho_p.size == self.n3
        xi_f = None if xi_f is None else _f64(xi_f)
        xi_g = None if xi_g is None else _f64(xi_g)
        if xi_f is not None:
            assert xi_f.size == 27 * self.n3
        if xi_g is not None:
            assert xi_g.size == 27 * self.n3
        lib().orc_init_fields(self._h, _dp(rho), _dp(u), _dp(rho_p), _dp(xi_f), _dp(xi_g),
                              float(amp))

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def populations(self):
        f = np.empty(len(self.wf) * self.n3)
        g = np.empty(len(self.wg) * self.n3)
        lib().orc_get_populations(self._h, _dp(f), _dp(g))
        return f.reshape(len(self.wf), self.n3), g.reshape(len(self.wg), self.n3)

    def set_populations(self, f, g):
        f, g = _f64(f), _f64(g)
        assert f.size == len(self.wf) * self.n3 and g.size == len(self.wg) * self.n3
        lib().orc_set_populations(self._h, _dp(f), _dp(g))

    def fields(self):
        rho = np.empty(self.n3)
        u = np.empty(3 * self.n3)
        rho_p = np.empty(self.n3)
        lib().orc_get_fields(self._h, _dp(rho), _dp(u), _dp(rho_p))
        return rho, u.reshape(3, self.n3), rho_p

    def diagnostics(self) -> dict:
        out = np.zeros(len(DIAG_NAMES))
        rc = lib().orc_diagnostics(self._h, _dp(out))
        if rc != 0:
            raise MemoryError("oracle diagnostics failed")
        d = dict(zip(DIAG_NAMES, out.tolist()))
        d["step"] = self.step_count
        return d
