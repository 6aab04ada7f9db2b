"""Long-window diagnostics series of the CUDA path: FP32 against the FP64
oracle, and FP16/BF16 deviation storage judged by the library's storage rule
(lbm_storage_rule) through the dissipation peaks (Section 3.3, Eqs. 22-26).

 - 64^3, D3Q27xD3Q19, Shan-Chen, Re 200 (the n/Re of the 256^3 Re 800
   workload, hence its tau_f), Fr 0.1, 5100 steps (t ~ 20 convective times),
   diagnostics every 25 steps (~t_c / 10): each storage against the oracle's
   series, stored in tests/golden by tests/golden/make_oracle_series.py.
 - 256^3, the same physics at Re 800 (the headline workload) for its full
   20000 steps with diagnostics every 100: FP16 and BF16 against the FP32 run
   on this GPU (no oracle at this size).

FP32 is held to the precision target at 1000 steps (E_k, E_p within 1e-5,
E_p relative to its window maximum) and to a bound derived from its measured
FP32 rounding drift over the whole window; the 16-bit storages are judged by
the 1 % rule, which keeps FP16 and demotes BF16 to FP32 on these series.
With LBM_TEST_REPORT set to a file name, every test appends its deviations to
that file as one JSON line.
"""
import importlib.util
import json
import os

import numpy as np
import pytest

import stgv_inputs as I
from paper_2605_14505_gb300 import lbm

pytestmark = pytest.mark.gpu

_spec = importlib.util.spec_from_file_location(
    "make_oracle_series", os.path.join(os.path.dirname(__file__), "golden", "make_oracle_series.py"))
G = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(G)

KEYS = ("Ek", "Ep", "eps_k", "eps_p")


def _report(record: dict):
    path = os.environ.get("LBM_TEST_REPORT")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps(record) + "\n")


def _gpu_series(n, pair, forcing, Re, Fr, Sc, U0, steps, every, seed, amp, storage):
    p = lbm.lbm_params_from_physics(n, n, n, pair, forcing, Re, Fr, Sc, U0)
    sim = lbm.Simulation(p, storage=storage)
    sim.init_fields(*I.tgv_fields(n, U0, seed=seed, noise_amp=amp))
    out = [sim.diagnostics()]
    for _ in range(steps // every):
        sim.step(every)
        out.append(sim.diagnostics())
    sim.close()
    return out


def _max_dev(a, b, key):
    ref = np.array([d[key] for d in b])
    got = np.array([d[key] for d in a])
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


NAME64 = "stgv64_re200_fr01_sc"


@pytest.fixture(scope="module")
def oracle64():
    return G.read(NAME64)


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_64cubed_series_against_the_oracle(oracle64, storage):
    n, (qf, qg), forcing, Re, Fr, Sc, U0, steps, every, seed, amp = G.SERIES[NAME64]
    gpu = _gpu_series(n, f"{qf}x{qg}", forcing, Re, Fr, Sc, U0, steps, every, seed, amp, storage)
    assert [d["step"] for d in gpu] == [d["step"] for d in oracle64]
    rep = lbm.lbm_storage_rule(oracle64, gpu, storage, 0.01)
    devs = {k: _max_dev(gpu, oracle64, k) for k in KEYS}
    k1000 = 1000 // every
    ep_max = max(d["Ep"] for d in oracle64[: k1000 + 1])
    at1000 = {"Ek": abs(gpu[k1000]["Ek"] - oracle64[k1000]["Ek"]) / oracle64[k1000]["Ek"],
              "Ep": abs(gpu[k1000]["Ep"] - oracle64[k1000]["Ep"]) / ep_max}
    _report({"test": "64cubed_vs_oracle", "storage": storage, "max_dev": devs, "at_step_1000": at1000,
             "rule": rep})
    if storage == "fp32":
        assert at1000["Ek"] <= 1e-5 and at1000["Ep"] <= 1e-5, at1000
        for k in KEYS:
            assert devs[k] <= 1e-4, (k, devs)
        assert rep["selected"] == "fp32"
    elif storage == "fp16":
        assert rep["pass"] and rep["selected"] == "fp16", rep
    else:
        assert not rep["pass"] and rep["selected"] == "fp32", rep


@pytest.fixture(scope="module")
def c2_fp32():
    return _gpu_series(256, "27x19", "sc", 800.0, 0.1, 1.0, 0.04, 20000, 100, 1, 1e-3, "fp32")


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_256cubed_workload_series_16bit_against_fp32(c2_fp32, storage):
    got = _gpu_series(256, "27x19", "sc", 800.0, 0.1, 1.0, 0.04, 20000, 100, 1, 1e-3, storage)
    rep = lbm.lbm_storage_rule(c2_fp32, got, storage, 0.01)
    devs = {k: _max_dev(got, c2_fp32, k) for k in KEYS}
    _report({"test": "256cubed_vs_fp32", "storage": storage, "max_dev": devs, "rule": rep})
    assert all(np.isfinite(d["Ek"]) for d in got)
    if storage == "fp16":
        assert rep["pass"] and rep["selected"] == "fp16", rep
    else:
        assert rep["selected"] == "fp32", rep


NAME64P = "stgv64_paper_re1600_fr1_sc"


@pytest.fixture(scope="module")
def oracle64p():
    return G.read(NAME64P)


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_64cubed_paper_parameters_against_the_oracle(oracle64p, storage):
    """The paper's parameters (Re0 1600, Sc 0.7, Ma 0.1, Fr0 1; Section 2.4) at
    64^3 to t ~ 30: the Taylor-Green vortex breaks down into turbulence and
    the total dissipation peaks twice (Section 3.3). Here tau_f - 1/2 is
    1.1e-3, 5.5 times smaller than in the workloads. FP32 is held to the
    precision target at step 1008 (t ~ 5.7, before the breakdown): measured
    E_k / E_p error 5.4e-7 / 5.9e-7, bound 1e-5; over the turbulent window
    (where the trajectories separate) max 7.1e-6 on eps_k, bound 1e-4. FP16
    is kept by the 1 % rule against the FP64 oracle through the peaks; BF16
    is demoted."""
    n, (qf, qg), forcing, Re, Fr, Sc, U0, steps, every, seed, amp = G.SERIES[NAME64P]
    gpu = _gpu_series(n, f"{qf}x{qg}", forcing, Re, Fr, Sc, U0, steps, every, seed, amp, storage)
    assert [d["step"] for d in gpu] == [d["step"] for d in oracle64p]
    rep = lbm.lbm_storage_rule(oracle64p, gpu, storage, 0.01)
    devs = {k: _max_dev(gpu, oracle64p, k) for k in KEYS}
    k1000 = round(1000 / every)
    ep_max = max(d["Ep"] for d in oracle64p[: k1000 + 1])
    at1000 = {"step": oracle64p[k1000]["step"],
              "Ek": abs(gpu[k1000]["Ek"] - oracle64p[k1000]["Ek"]) / oracle64p[k1000]["Ek"],
              "Ep": abs(gpu[k1000]["Ep"] - oracle64p[k1000]["Ep"]) / ep_max}
    _report({"test": "64cubed_paper_vs_oracle", "storage": storage, "max_dev": devs, "at_step_1000": at1000,
             "rule": rep})
    assert all(np.isfinite(d["Ek"]) for d in gpu)
    if storage == "fp32":
        assert at1000["Ek"] <= 1e-5 and at1000["Ep"] <= 1e-5, at1000
        for k in KEYS:
            assert devs[k] <= 1e-4, (k, devs)
    elif storage == "fp16":
        assert rep["pass"] and rep["selected"] == "fp16", rep
    else:
        assert not rep["pass"] and rep["selected"] == "fp32", rep


# The 128^3 workload (both stencil pairs x Guo / Shan-Chen x Fr 0.5 / 0.1, Re 400,
# 5000 steps, diagnostics every 50) against its stored FP64 oracle series.
C1_NAMES = sorted(n for n in G.SERIES if n.startswith("c1_") and os.path.exists(G.path_of(n)))


@pytest.mark.parametrize("name", C1_NAMES or ["c1_128_q19q7_guo_fr0.5"])
@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_128cubed_workload_series_against_the_oracle(name, storage):
    """FP32: E_k and E_p within 1e-5 at step 1000 (E_p relative to its window
    maximum) and every diagnostics quantity within 1e-4 of the oracle over the
    5000 steps; FP16: kept by the 1 % storage rule against the FP64 series."""
    n, (qf, qg), forcing, Re, Fr, Sc, U0, steps, every, seed, amp = G.SERIES[name]
    ref = G.read(name)
    gpu = _gpu_series(n, f"{qf}x{qg}", forcing, Re, Fr, Sc, U0, steps, every, seed, amp, storage)
    assert [d["step"] for d in gpu] == [d["step"] for d in ref]
    rep = lbm.lbm_storage_rule(ref, gpu, storage, 0.01)
    devs = {k: _max_dev(gpu, ref, k) for k in KEYS}
    k1000 = 1000 // every
    ep_max = max(d["Ep"] for d in ref[: k1000 + 1])
    at1000 = {"Ek": abs(gpu[k1000]["Ek"] - ref[k1000]["Ek"]) / ref[k1000]["Ek"],
              "Ep": abs(gpu[k1000]["Ep"] - ref[k1000]["Ep"]) / ep_max}
    _report({"test": "128cubed_vs_oracle", "series": name, "storage": storage, "max_dev": devs,
             "at_step_1000": at1000, "rule": rep})
    if storage == "fp32":
        assert at1000["Ek"] <= 1e-5 and at1000["Ep"] <= 1e-5, at1000
        for k in KEYS:
            assert devs[k] <= 1e-4, (k, devs)
    else:
        assert rep["pass"] and rep["selected"] == "fp16", rep
