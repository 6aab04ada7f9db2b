"""The 16-bit storage rule of the C library (lbm_storage_rule), on synthetic
series. It is host logic (no device work), so these tests run without a GPU;
the GPU tests apply it to measured FP16/BF16 series (tests/test_gpu_series.py).

The rule keeps a 16-bit storage only while E_k, E_p, eps_k and eps_p stay
within tol of the reference series (relative to each series' maximum) and the
total dissipation eps_k + eps_p at the reference's two highest peaks (the
double peak of Section 3.3) within tol of each peak's height; otherwise FP32.
"""
import math

import numpy as np
import pytest

from paper_2605_14505_gb300 import lbm


def _series(steps, eps_k, scale=1.0):
    return [{"step": int(s), "Ek": 1e-3 * scale * (1 + 0.1 * i / len(steps)),
             "Ep": 2e-5 * scale * math.sin(0.3 * i) ** 2, "eps_k": float(e) * scale,
             "eps_p": 0.1 * float(e) * scale} for i, (s, e) in enumerate(zip(steps, eps_k))]


def _double_peak(t):
    # two bumps: heights 1.0 at t = 11.5 and 0.8 at t = 16.5 (the second is lower)
    return 1e-6 * (0.1 + np.exp(-((t - 11.5) / 1.2) ** 2) + 0.8 * np.exp(-((t - 16.5) / 1.0) ** 2))


def test_identical_series_pass_and_the_double_peak_is_found():
    t = np.linspace(0, 20, 201)
    ref = _series(np.arange(201) * 25, _double_peak(t))
    rep = lbm.lbm_storage_rule(ref, ref, "fp16", 0.01)
    assert rep["pass"] and rep["selected"] == "fp16"
    assert rep["dev_Ek"] == 0 and rep["dev_eps_k"] == 0 and rep["dev_peak1"] == 0
    assert rep["step_peak1"] == 115 * 25 and rep["step_peak2"] == 165 * 25


@pytest.mark.parametrize("key", ["Ek", "Ep", "eps_k", "eps_p"])
def test_one_quantity_beyond_the_bound_falls_back_to_fp32(key):
    t = np.linspace(0, 20, 201)
    ref = _series(np.arange(201) * 25, _double_peak(t))
    cand = [dict(d) for d in ref]
    scale = max(abs(d[key]) for d in ref)
    cand[40][key] += 0.02 * scale          # 2 % of the series maximum at one sample
    rep = lbm.lbm_storage_rule(ref, cand, "bf16", 0.01)
    assert not rep["pass"] and rep["selected"] == "fp32"
    assert rep["dev_" + key] == pytest.approx(0.02, rel=1e-12)
    # within the bound: kept
    cand[40][key] = ref[40][key] + 0.005 * scale
    rep = lbm.lbm_storage_rule(ref, cand, "bf16", 0.01)
    assert rep["pass"] and rep["selected"] == "bf16"


def test_second_peak_is_judged_against_its_own_height():
    """A drift of 1.1 % of the second (lower) peak's height stays under 1 % of
    the series maximum, yet it breaks the bound on that peak."""
    t = np.linspace(0, 20, 201)
    ref = _series(np.arange(201) * 25, _double_peak(t))
    k2 = 165
    cand = [dict(d) for d in ref]
    # shift eps_k at the second peak so that eps_k + eps_p moves by 1.1 % of that peak
    e2 = ref[k2]["eps_k"] + ref[k2]["eps_p"]
    cand[k2]["eps_k"] += 0.011 * e2
    emax = max(d["eps_k"] for d in ref)
    assert 0.011 * e2 / emax < 0.01       # within the series bound
    rep = lbm.lbm_storage_rule(ref, cand, "fp16", 0.01)
    assert rep["dev_eps_k"] < 0.01 and rep["dev_peak2"] == pytest.approx(0.011, rel=1e-9)
    assert not rep["pass"] and rep["selected"] == "fp32"


def test_non_finite_candidate_fails_and_bad_input_is_rejected():
    t = np.linspace(0, 20, 101)
    ref = _series(np.arange(101) * 50, _double_peak(t))
    cand = [dict(d) for d in ref]
    cand[7]["eps_p"] = float("nan")
    rep = lbm.lbm_storage_rule(ref, cand, "fp16", 0.01)
    assert rep["selected"] == "fp32" and math.isinf(rep["dev_eps_p"])
    # steps must match
    cand = [dict(d) for d in ref]
    cand[3]["step"] += 1
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_storage_rule(ref, cand, "fp16", 0.01)
    assert ei.value.code == -1
    with pytest.raises(lbm.LbmError):
        lbm.lbm_storage_rule(ref, ref, "fp16", 0.0)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_storage_rule(ref, ref, 7, 0.01)


def test_monotone_series_has_no_peak_check():
    steps = np.arange(50) * 10
    ref = _series(steps, np.linspace(1e-7, 1e-6, 50))
    rep = lbm.lbm_storage_rule(ref, ref, "fp16", 0.01)
    assert rep["step_peak1"] == -1 and rep["step_peak2"] == -1
    assert math.isnan(rep["dev_peak1"]) and rep["pass"]
