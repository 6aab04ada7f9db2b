"""Thin ctypes binding of the C ABI in ``include/lbm.h`` (same function names).

Every step of the lattice Boltzmann update runs in ``liblbm.so`` on the GPU;
this module only marshals arguments, raises :class:`LbmError` on a non-zero
status, and (in :class:`Simulation`) hands the library device memory and a
CUDA stream taken from PyTorch. There is no CPU fallback: if the library is
missing or cannot load, importing the binding raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "lbm.h")

LBM_OK = 0
STATUS = {
    -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA", -4: "LBM_ETIMEOUT",
    -5: "LBM_ENONFINITE", -6: "LBM_EUNSUPPORTED", -7: "LBM_ESTATE",
}
PAIRS = {
    "27x19": 0, "19x7": 1, "27x27": 2, "19x19": 3, "19x15": 4, "15x7": 5, "7x27": 6,
}
PAIR_Q = {0: (27, 19), 1: (19, 7), 2: (27, 27), 3: (19, 19), 4: (19, 15), 5: (15, 7), 6: (7, 27)}
FORCINGS = {"guo": 0, "sc": 1, "shan_chen": 1, "edm": 2, "hcz": 3}
STORAGES = {"fp32": 0, "fp16": 1, "bf16": 2}
SCALAR_MODES = {"printed": 0, "chai_shi": 1}


class LbmError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{STATUS.get(code, code)}: {message}")
        self.code = code


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("pair", ctypes.c_int32), ("forcing", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("scalar_mode", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("tau_f", ctypes.c_double), ("tau_g", ctypes.c_double), ("G", ctypes.c_double),
        ("beta", ctypes.c_double), ("rho0", ctypes.c_double), ("sc_shift", ctypes.c_double),
        ("U0", ctypes.c_double), ("L", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


class lbm_diag(ctypes.Structure):
    _fields_ = [
        ("Ek", ctypes.c_double), ("Ep", ctypes.c_double), ("eps_k", ctypes.c_double),
        ("eps_p", ctypes.c_double), ("eps_k_curl", ctypes.c_double),
        ("mass_f", ctypes.c_double), ("mass_g", ctypes.c_double),
        ("mom", ctypes.c_double * 3), ("umax", ctypes.c_double), ("step", ctypes.c_int64),
        ("t", ctypes.c_double), ("Ek_phys", ctypes.c_double), ("Ep_phys", ctypes.c_double),
        ("eps_k_phys", ctypes.c_double), ("eps_p_phys", ctypes.c_double),
        ("eps_k_curl_phys", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {
            "Ek": self.Ek, "Ep": self.Ep, "eps_k": self.eps_k, "eps_p": self.eps_p,
            "eps_k_curl": self.eps_k_curl, "mass_f": self.mass_f, "mass_g": self.mass_g,
            "mom_x": self.mom[0], "mom_y": self.mom[1], "mom_z": self.mom[2],
            "umax": self.umax, "step": int(self.step),
            "t": self.t, "Ek_phys": self.Ek_phys, "Ep_phys": self.Ep_phys,
            "eps_k_phys": self.eps_k_phys, "eps_p_phys": self.eps_p_phys,
            "eps_k_curl_phys": self.eps_k_curl_phys,
        }


class lbm_storage_report(ctypes.Structure):
    _fields_ = [
        ("dev_Ek", ctypes.c_double), ("dev_Ep", ctypes.c_double), ("dev_eps_k", ctypes.c_double),
        ("dev_eps_p", ctypes.c_double), ("dev_peak1", ctypes.c_double), ("dev_peak2", ctypes.c_double),
        ("step_peak1", ctypes.c_int64), ("step_peak2", ctypes.c_int64),
        ("selected", ctypes.c_int32), ("pass_", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        names = {v: k for k, v in STORAGES.items()}
        return {
            "dev_Ek": self.dev_Ek, "dev_Ep": self.dev_Ep, "dev_eps_k": self.dev_eps_k,
            "dev_eps_p": self.dev_eps_p, "dev_peak1": self.dev_peak1, "dev_peak2": self.dev_peak2,
            "step_peak1": int(self.step_peak1), "step_peak2": int(self.step_peak2),
            "selected": names.get(self.selected, self.selected), "pass": bool(self.pass_),
        }


_H = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "lbm_last_error": ([], ctypes.c_char_p),
    "lbm_version": ([], ctypes.c_char_p),
    "lbm_velocity_set": ([ctypes.c_int, ctypes.POINTER(ctypes.c_int), _DP, _DP], ctypes.c_int),
    "lbm_params_from_physics": ([ctypes.POINTER(lbm_params), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double], ctypes.c_int),
    "lbm_create": ([ctypes.POINTER(_H), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                    ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                    ctypes.c_double], ctypes.c_int),
    "lbm_create_params": ([ctypes.POINTER(_H), ctypes.POINTER(lbm_params)], ctypes.c_int),
    "lbm_get_params": ([_H, ctypes.POINTER(lbm_params)], ctypes.c_int),
    "lbm_set_storage": ([_H, ctypes.c_int], ctypes.c_int),
    "lbm_set_stream": ([_H, ctypes.c_void_p], ctypes.c_int),
    "lbm_required_bytes": ([_H, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "lbm_attach": ([_H, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "lbm_init_tgv": ([_H, ctypes.c_uint64, ctypes.c_double], ctypes.c_int),
    "lbm_init_fields": ([_H, _DP, _DP, _DP, _DP, _DP, ctypes.c_double], ctypes.c_int),
    "lbm_step": ([_H, ctypes.c_int64], ctypes.c_int),
    "lbm_synchronize": ([_H], ctypes.c_int),
    "lbm_diagnostics": ([_H, ctypes.POINTER(lbm_diag)], ctypes.c_int),
    "lbm_step_diagnostics": ([_H, ctypes.c_int64, ctypes.POINTER(lbm_diag)], ctypes.c_int),
    "lbm_prefetch_fields": ([_H, _DP, _DP, _DP], ctypes.c_int),
    "lbm_init_prefetched": ([_H], ctypes.c_int),
    "lbm_diagnostics_noalloc": ([_H, ctypes.POINTER(lbm_diag)], ctypes.c_int),
    "lbm_storage_rule": ([ctypes.POINTER(lbm_diag), ctypes.POINTER(lbm_diag), ctypes.c_int64, ctypes.c_int,
                          ctypes.c_double, ctypes.POINTER(lbm_storage_report)], ctypes.c_int),
    "lbm_get_fields": ([_H, _DP, _DP, _DP], ctypes.c_int),
    "lbm_get_fields_device": ([_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "lbm_get_populations": ([_H, _DP, _DP], ctypes.c_int),
    "lbm_set_populations": ([_H, _DP, _DP], ctypes.c_int),
    "lbm_sample_populations": ([_H, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, _DP, _DP],
                               ctypes.c_int),
    "lbm_step_count": ([_H, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "lbm_set_block": ([_H, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "lbm_get_block": ([_H, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "lbm_autotune": ([_H, ctypes.c_int, _DP], ctypes.c_int),
    "lbm_set_graphs": ([_H, ctypes.c_int], ctypes.c_int),
    "lbm_set_slab": ([_H, ctypes.c_int], ctypes.c_int),
    "lbm_halo_bytes": ([_H, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "lbm_halo_pack": ([_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "lbm_halo_unpack": ([_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "lbm_set_pairing": ([_H, ctypes.c_int], ctypes.c_int),
    "lbm_set_tile_staging": ([_H, ctypes.c_int], ctypes.c_int),
    "lbm_uses_tile_staging": ([_H, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "lbm_set_stage_test": ([_H, ctypes.c_uint, ctypes.c_uint], ctypes.c_int),
    "lbm_destroy": ([_H], ctypes.c_int),
    "lbm_batch_create": ([ctypes.POINTER(_H), ctypes.POINTER(lbm_params), ctypes.c_int], ctypes.c_int),
    "lbm_batch_count": ([_H, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "lbm_batch_instance": ([_H, ctypes.c_int, ctypes.POINTER(_H)], ctypes.c_int),
    "lbm_batch_set_stream": ([_H, ctypes.c_void_p], ctypes.c_int),
    "lbm_batch_set_mode": ([_H, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "lbm_batch_set_block": ([_H, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "lbm_batch_get_config": ([_H] + [ctypes.POINTER(ctypes.c_int)] * 4, ctypes.c_int),
    "lbm_batch_init_tgv": ([_H, ctypes.c_uint64, ctypes.c_double], ctypes.c_int),
    "lbm_batch_step": ([_H, ctypes.c_int64], ctypes.c_int),
    "lbm_batch_synchronize": ([_H], ctypes.c_int),
    "lbm_batch_diagnostics": ([_H, ctypes.POINTER(lbm_diag)], ctypes.c_int),
    "lbm_batch_autotune": ([_H, ctypes.c_int, _DP], ctypes.c_int),
    "lbm_batch_set_barrier_test": ([_H, ctypes.c_uint, ctypes.c_uint], ctypes.c_int),
    "lbm_batch_set_flow_nodes": ([_H, ctypes.c_int], ctypes.c_int),
    "lbm_batch_partition": ([ctypes.POINTER(lbm_params), ctypes.c_int, ctypes.c_int,
                             ctypes.POINTER(ctypes.c_int32), _DP], ctypes.c_int),
    "lbm_batch_get_flow_nodes": ([_H, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "lbm_batch_destroy": ([_H], ctypes.c_int),
}
BATCH_MODES = {"persistent": 0, "per_step": 1, "instances": 2}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(
                f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def header_functions(path: str = HEADER_PATH) -> list[str]:
    """Names of the functions declared in include/lbm.h."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def _check(rc: int):
    if rc != LBM_OK:
        raise LbmError(rc, load_library().lbm_last_error().decode())
    return rc


def _dp(a):
    return None if a is None else a.ctypes.data_as(_DP)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- same-name wrappers -------------------------------------------------------

def lbm_last_error() -> str:
    return load_library().lbm_last_error().decode()


def lbm_version() -> str:
    return load_library().lbm_version().decode()


def lbm_velocity_set(q: int):
    e = np.zeros(81, dtype=np.int32)
    w = np.zeros(27)
    cs2 = ctypes.c_double()
    n = load_library().lbm_velocity_set(q, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                                        ctypes.byref(cs2))
    if n < 0:
        _check(n)
    return e[: 3 * n].reshape(n, 3).copy(), w[:n].copy(), cs2.value


def _enum(v, table):
    return table[v] if isinstance(v, str) else int(v)


def lbm_params_from_physics(nx, ny, nz, pair, forcing, Re, Fr, Pr, U0) -> lbm_params:
    p = lbm_params()
    _check(load_library().lbm_params_from_physics(ctypes.byref(p), nx, ny, nz, _enum(pair, PAIRS),
                                                  _enum(forcing, FORCINGS), Re, Fr, Pr, U0))
    return p


def lbm_create(nx, ny, nz, pair, forcing, Re, Fr, Pr, U0) -> ctypes.c_void_p:
    h = _H()
    _check(load_library().lbm_create(ctypes.byref(h), nx, ny, nz, _enum(pair, PAIRS),
                                     _enum(forcing, FORCINGS), Re, Fr, Pr, U0))
    return h


def lbm_create_params(p: lbm_params) -> ctypes.c_void_p:
    h = _H()
    _check(load_library().lbm_create_params(ctypes.byref(h), ctypes.byref(p)))
    return h


def lbm_get_params(h) -> lbm_params:
    p = lbm_params()
    _check(load_library().lbm_get_params(h, ctypes.byref(p)))
    return p


def lbm_set_storage(h, storage):
    _check(load_library().lbm_set_storage(h, _enum(storage, STORAGES)))


def lbm_set_stream(h, stream_ptr: int):
    _check(load_library().lbm_set_stream(h, ctypes.c_void_p(stream_ptr)))


def lbm_required_bytes(h) -> int:
    n = ctypes.c_size_t()
    _check(load_library().lbm_required_bytes(h, ctypes.byref(n)))
    return n.value


def lbm_attach(h, device_ptr: int, nbytes: int):
    _check(load_library().lbm_attach(h, ctypes.c_void_p(device_ptr), nbytes))


def lbm_init_tgv(h, seed: int = 0, noise_amp: float = 0.0):
    _check(load_library().lbm_init_tgv(h, seed, noise_amp))


def lbm_init_fields(h, rho, u, rho_p, xi_f=None, xi_g=None, amp: float = 0.0):
    rho, u, rho_p = _f64(rho), _f64(u), _f64(rho_p)
    xi_f = None if xi_f is None else _f64(xi_f)
    xi_g = None if xi_g is None else _f64(xi_g)
    _check(load_library().lbm_init_fields(h, _dp(rho), _dp(u), _dp(rho_p), _dp(xi_f), _dp(xi_g), amp))


def _host_f64_ptr(x):
    """Pointer to a C-contiguous float64 host array (numpy, or a CPU torch
    tensor, e.g. in pinned memory) without copying it."""
    if hasattr(x, "data_ptr"):
        if x.dtype.__str__() != "torch.float64" or x.is_cuda or not x.is_contiguous():
            raise ValueError("expected a contiguous CPU float64 tensor")
        return ctypes.cast(x.data_ptr(), _DP)
    if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
        raise ValueError("expected a C-contiguous float64 array")
    return x.ctypes.data_as(_DP)


def lbm_prefetch_fields(h, rho, u, rho_p):
    """Start the host-to-device copies of the next state's fields (see the C
    header); the arrays must stay alive and unchanged until
    lbm_init_prefetched returns."""
    _check(load_library().lbm_prefetch_fields(h, _host_f64_ptr(rho), _host_f64_ptr(u), _host_f64_ptr(rho_p)))


def lbm_init_prefetched(h):
    _check(load_library().lbm_init_prefetched(h))


def lbm_step(h, nsteps: int):
    _check(load_library().lbm_step(h, int(nsteps)))


def lbm_synchronize(h):
    _check(load_library().lbm_synchronize(h))


def lbm_diagnostics(h, allow_nonfinite: bool = False) -> dict:
    d = lbm_diag()
    rc = load_library().lbm_diagnostics(h, ctypes.byref(d))
    if not (allow_nonfinite and rc == -5):
        _check(rc)
    return d.as_dict()


def lbm_step_diagnostics(h, nsteps: int, allow_nonfinite: bool = False) -> dict:
    """Diagnostics of the current state, reduced inside the first of `nsteps`
    steps, which then all run."""
    d = lbm_diag()
    rc = load_library().lbm_step_diagnostics(h, int(nsteps), ctypes.byref(d))
    if not (allow_nonfinite and rc == -5):
        _check(rc)
    return d.as_dict()


def lbm_diagnostics_noalloc(h) -> dict:
    """lbm_diagnostics without any device allocation (eps_p, eps_k_curl are NaN)."""
    d = lbm_diag()
    _check(load_library().lbm_diagnostics_noalloc(h, ctypes.byref(d)))
    return d.as_dict()


_DIAG_KEYS = ("Ek", "Ep", "eps_k", "eps_p", "eps_k_curl", "mass_f", "mass_g", "umax", "t", "Ek_phys",
              "Ep_phys", "eps_k_phys", "eps_p_phys", "eps_k_curl_phys")


def _diag_array(series):
    """lbm_diag records from dicts (as returned by the diagnostics wrappers,
    or by the oracle's view: missing fields are NaN)."""
    arr = (lbm_diag * len(series))()
    for rec, d in zip(arr, series):
        for k in _DIAG_KEYS:
            setattr(rec, k, float(d.get(k, float("nan"))))
        for a, k in enumerate(("mom_x", "mom_y", "mom_z")):
            rec.mom[a] = float(d.get(k, float("nan")))
        rec.step = int(d["step"])
    return arr


def lbm_storage_rule(reference, candidate, candidate_storage, tol: float = 0.01) -> dict:
    """The 16-bit storage rule of the C library on two diagnostics series
    (lists of dicts with the same steps). Returns the report; report["selected"]
    is the storage to use ("fp32" when the candidate misses the bound)."""
    if len(reference) != len(candidate):
        raise ValueError("the two series must have the same samples")
    ref, cand = _diag_array(reference), _diag_array(candidate)
    rep = lbm_storage_report()
    rc = load_library().lbm_storage_rule(ref, cand, len(reference), _enum(candidate_storage, STORAGES),
                                         float(tol), ctypes.byref(rep))
    if rc < 0:
        _check(rc)
    return rep.as_dict()


def lbm_get_fields(h, n3: int):
    rho = np.empty(n3)
    u = np.empty(3 * n3)
    rho_p = np.empty(n3)
    _check(load_library().lbm_get_fields(h, _dp(rho), _dp(u), _dp(rho_p)))
    return rho, u.reshape(3, n3), rho_p


def lbm_get_fields_device(h, rho_ptr, u_ptr, rho_p_ptr):
    """Device pointers (ints, or None) of FP64 buffers of n3, 3*n3, n3 values;
    the fields are written asynchronously on the handle's stream."""
    _check(load_library().lbm_get_fields_device(h, rho_ptr, u_ptr, rho_p_ptr))


def lbm_get_populations(h, qf: int, qg: int, n3: int):
    f = np.empty(qf * n3)
    g = np.empty(qg * n3)
    _check(load_library().lbm_get_populations(h, _dp(f), _dp(g)))
    return f.reshape(qf, n3), g.reshape(qg, n3)


def lbm_sample_populations(h, nodes, qf: int, qg: int):
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    f = np.empty(len(nodes) * qf)
    g = np.empty(len(nodes) * qg)
    _check(load_library().lbm_sample_populations(
        h, nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(nodes), _dp(f), _dp(g)))
    return f.reshape(len(nodes), qf), g.reshape(len(nodes), qg)


def lbm_set_populations(h, f, g):
    f, g = _f64(f), _f64(g)
    _check(load_library().lbm_set_populations(h, _dp(f), _dp(g)))


def lbm_step_count(h) -> int:
    s = ctypes.c_int64()
    _check(load_library().lbm_step_count(h, ctypes.byref(s)))
    return s.value


def lbm_set_block(h, bx: int, by: int):
    _check(load_library().lbm_set_block(h, bx, by))


def lbm_get_block(h):
    bx, by = ctypes.c_int(), ctypes.c_int()
    _check(load_library().lbm_get_block(h, ctypes.byref(bx), ctypes.byref(by)))
    return bx.value, by.value


def lbm_autotune(h, reps: int = 3) -> float:
    ms = ctypes.c_double()
    _check(load_library().lbm_autotune(h, reps, ctypes.byref(ms)))
    return ms.value


PAIRING = {"off": 0, "all": 1, "even": 2}


def lbm_set_pairing(h, mode):
    """mode: "off", "all", "even" (or 0/1/2; True/False mean "all"/"off")."""
    if isinstance(mode, str):
        mode = PAIRING[mode]
    _check(load_library().lbm_set_pairing(h, int(mode)))


def lbm_set_tile_staging(h, enable: bool):
    _check(load_library().lbm_set_tile_staging(h, 1 if enable else 0))


def lbm_uses_tile_staging(h) -> int:
    w = ctypes.c_int(0)
    _check(load_library().lbm_uses_tile_staging(h, ctypes.byref(w)))
    return w.value


def lbm_set_stage_test(h, extra_tx_bytes: int, spin_limit: int):
    _check(load_library().lbm_set_stage_test(h, int(extra_tx_bytes), int(spin_limit)))


def lbm_set_slab(h, enable: bool):
    _check(load_library().lbm_set_slab(h, 1 if enable else 0))


def lbm_halo_bytes(h) -> int:
    n = ctypes.c_size_t()
    _check(load_library().lbm_halo_bytes(h, ctypes.byref(n)))
    return n.value


def lbm_halo_pack(h, phase: int, to_lower: int, to_upper: int):
    _check(load_library().lbm_halo_pack(h, int(phase), ctypes.c_void_p(to_lower), ctypes.c_void_p(to_upper)))


def lbm_halo_unpack(h, phase: int, from_lower: int, from_upper: int):
    _check(load_library().lbm_halo_unpack(h, int(phase), ctypes.c_void_p(from_lower), ctypes.c_void_p(from_upper)))


def lbm_set_graphs(h, enable: bool):
    _check(load_library().lbm_set_graphs(h, 1 if enable else 0))


def lbm_destroy(h):
    if h:
        _check(load_library().lbm_destroy(h))


# ---- convenience object ---------------------------------------------------------

class Simulation:
    """One lattice on the current CUDA device. The population store is a
    PyTorch allocation handed to the library (lbm_attach) and all work goes to
    a PyTorch-created CUDA stream (lbm_set_stream)."""

    def __init__(self, params: lbm_params, storage=None, torch_memory: bool = True):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        p = lbm_params()
        ctypes.pointer(p)[0] = params
        if storage is not None:
            p.storage = _enum(storage, STORAGES)
        self.params = p
        self.qf, self.qg = PAIR_Q[p.pair]
        self.n3 = p.nx * p.ny * p.nz
        self.h = lbm_create_params(p)
        self.stream = torch.cuda.Stream()
        lbm_set_stream(self.h, self.stream.cuda_stream)
        self._store = None
        if torch_memory:
            nbytes = lbm_required_bytes(self.h)
            self._store = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            lbm_attach(self.h, self._store.data_ptr(), nbytes)

    @classmethod
    def from_physics(cls, n, pair="27x19", forcing="sc", Re=800.0, Fr=0.1, Pr=1.0, U0=0.04,
                     storage="fp32", **kw):
        return cls(lbm_params_from_physics(n, n, n, pair, forcing, Re, Fr, Pr, U0), storage=storage, **kw)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None
        self._store = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_tgv(self, seed=0, noise_amp=0.0):
        lbm_init_tgv(self.h, seed, noise_amp)

    def init_fields(self, rho, u, rho_p, xi_f=None, xi_g=None, amp=0.0):
        lbm_init_fields(self.h, rho, u, rho_p, xi_f, xi_g, amp)

    def step(self, n=1):
        lbm_step(self.h, n)

    def synchronize(self):
        lbm_synchronize(self.h)

    def diagnostics(self, allow_nonfinite=False) -> dict:
        return lbm_diagnostics(self.h, allow_nonfinite)

    def step_diagnostics(self, n, allow_nonfinite=False) -> dict:
        return lbm_step_diagnostics(self.h, n, allow_nonfinite)

    def fields(self):
        return lbm_get_fields(self.h, self.n3)

    def fields_device(self):
        """(rho, u[3, n3], rho') as FP64 CUDA tensors, written by the library
        on its stream (which this waits for)."""
        import torch

        rho = torch.empty(self.n3, dtype=torch.float64, device="cuda")
        u = torch.empty((3, self.n3), dtype=torch.float64, device="cuda")
        rp = torch.empty(self.n3, dtype=torch.float64, device="cuda")
        lbm_get_fields_device(self.h, rho.data_ptr(), u.data_ptr(), rp.data_ptr())
        self.synchronize()
        return rho, u, rp

    def populations(self):
        return lbm_get_populations(self.h, self.qf, self.qg, self.n3)

    def set_populations(self, f, g):
        lbm_set_populations(self.h, f, g)

    def sample_populations(self, nodes):
        return lbm_sample_populations(self.h, nodes, self.qf, self.qg)

    @property
    def step_count(self) -> int:
        return lbm_step_count(self.h)

    def velocity_sets(self):
        return lbm_velocity_set(self.qf), lbm_velocity_set(self.qg)


# ---- batched instances -------------------------------------------------------

def lbm_batch_create(params_list) -> ctypes.c_void_p:
    arr = (lbm_params * len(params_list))(*params_list)
    b = _H()
    _check(load_library().lbm_batch_create(ctypes.byref(b), arr, len(params_list)))
    return b


def lbm_batch_count(b) -> int:
    c = ctypes.c_int()
    _check(load_library().lbm_batch_count(b, ctypes.byref(c)))
    return c.value


def lbm_batch_instance(b, i: int) -> ctypes.c_void_p:
    h = _H()
    _check(load_library().lbm_batch_instance(b, i, ctypes.byref(h)))
    return h


def lbm_batch_set_stream(b, stream_ptr: int):
    _check(load_library().lbm_batch_set_stream(b, ctypes.c_void_p(stream_ptr)))


def lbm_batch_set_mode(b, mode, steps_per_launch: int = 100):
    _check(load_library().lbm_batch_set_mode(b, _enum(mode, BATCH_MODES), steps_per_launch))


def lbm_batch_set_block(b, bx: int, by: int):
    _check(load_library().lbm_batch_set_block(b, bx, by))


def lbm_batch_get_config(b) -> dict:
    v = [ctypes.c_int() for _ in range(4)]
    _check(load_library().lbm_batch_get_config(b, *[ctypes.byref(x) for x in v]))
    return {"bx": v[0].value, "by": v[1].value, "mode": v[2].value, "grid": v[3].value}


def lbm_batch_init_tgv(b, seed: int = 0, noise_amp: float = 0.0):
    _check(load_library().lbm_batch_init_tgv(b, seed, noise_amp))


def lbm_batch_step(b, nsteps: int):
    _check(load_library().lbm_batch_step(b, int(nsteps)))


def lbm_batch_synchronize(b):
    _check(load_library().lbm_batch_synchronize(b))


def lbm_batch_diagnostics(b) -> list:
    n = lbm_batch_count(b)
    out = (lbm_diag * n)()
    _check(load_library().lbm_batch_diagnostics(b, out))
    return [d.as_dict() for d in out]


def lbm_batch_autotune(b, reps: int = 3) -> float:
    ms = ctypes.c_double()
    _check(load_library().lbm_batch_autotune(b, reps, ctypes.byref(ms)))
    return ms.value


def lbm_batch_set_barrier_test(b, extra_completions: int, spin_limit: int):
    _check(load_library().lbm_batch_set_barrier_test(b, extra_completions, spin_limit))


def lbm_batch_partition(params_list, nranks: int):
    """(owner list, imbalance): the rank of every instance (see the C header)."""
    arr = (lbm_params * len(params_list))(*params_list)
    owner = (ctypes.c_int32 * len(params_list))()
    imb = ctypes.c_double()
    _check(load_library().lbm_batch_partition(arr, len(params_list), int(nranks), owner, ctypes.byref(imb)))
    return list(owner), imb.value


def lbm_batch_set_flow_nodes(b, nodes: int):
    _check(load_library().lbm_batch_set_flow_nodes(b, int(nodes)))


def lbm_batch_get_flow_nodes(b) -> int:
    n = ctypes.c_int()
    _check(load_library().lbm_batch_get_flow_nodes(b, ctypes.byref(n)))
    return n.value


def lbm_batch_destroy(b):
    if b:
        _check(load_library().lbm_batch_destroy(b))
