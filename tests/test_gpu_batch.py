"""Batched instances (many lattices advanced together) against single-lattice
runs and the oracle, all three drivers, the 64-instance sweep, and the
persistent driver's timeout path (its dependency waits made to run out on
purpose, with a short poll limit: the kernel returns an error status and the
context stays usable)."""
import numpy as np
import pytest

import stgv_inputs as I
from paper_2605_14505_gb300 import lbm

from _helpers import oracle_for, slot_map

pytestmark = pytest.mark.gpu

SMALL = [
    (16, "27x19", "guo", 100.0, 0.5),
    (24, "19x7", "sc", 150.0, 0.2),
    (20, "27x19", "edm", 120.0, 1.0),
    (12, "19x7", "hcz", 80.0, 0.1),
    (40, "27x19", "sc", 200.0, 0.1),
]


def _params(n, pair, forcing, Re, Fr):
    return lbm.lbm_params_from_physics(n, n, n, pair, forcing, Re, Fr, 1.0, 0.04)


def _batch(specs, mode="persistent", steps_per_launch=7, block=None):
    b = lbm.lbm_batch_create([_params(*s) for s in specs])
    lbm.lbm_batch_set_mode(b, mode, steps_per_launch)
    if block:
        lbm.lbm_batch_set_block(b, *block)
    lbm.lbm_batch_init_tgv(b, seed=5, noise_amp=0.02)
    return b


def _pops(h, p):
    qf, qg = lbm.PAIR_Q[p.pair]
    return lbm.lbm_get_populations(h, qf, qg, p.nx * p.ny * p.nz)


def test_batch_matches_single_lattices():
    b = _batch(SMALL)
    lbm.lbm_batch_step(b, 33)
    lbm.lbm_batch_synchronize(b)
    for i, s in enumerate(SMALL):
        p = _params(*s)
        solo = lbm.Simulation(p)
        solo.init_tgv(seed=5, noise_amp=0.02)
        solo.step(33)
        fs, gs = solo.populations()
        fb, gb = _pops(lbm.lbm_batch_instance(b, i), p)
        scale_f = np.max(np.abs(fs - lbm.lbm_velocity_set(lbm.PAIR_Q[p.pair][0])[1][:, None]))
        # same per-node arithmetic; the compiler may contract differently in
        # the batched kernel, so allow FP32 rounding
        assert np.max(np.abs(fb - fs)) <= 1e-6 * scale_f, i
        assert np.max(np.abs(gb - gs)) <= 1e-6 * np.max(np.abs(gs)), i
        solo.close()
    lbm.lbm_batch_destroy(b)


def test_persistent_and_per_step_drivers_agree_bitwise():
    a = _batch(SMALL, "persistent", 10)
    c = _batch(SMALL, "per_step")
    for b in (a, c):
        lbm.lbm_batch_step(b, 131)  # graph replays + eager tail / 14 persistent launches
        lbm.lbm_batch_synchronize(b)
    for i, s in enumerate(SMALL):
        p = _params(*s)
        fa, ga = _pops(lbm.lbm_batch_instance(a, i), p)
        fc, gc = _pops(lbm.lbm_batch_instance(c, i), p)
        assert np.array_equal(fa, fc) and np.array_equal(ga, gc), i
    lbm.lbm_batch_destroy(a)
    lbm.lbm_batch_destroy(c)


def test_instance_driver_is_the_single_lattice_run():
    """The per-instance driver runs every instance's own single-lattice step
    kernel (one graph branch per instance): bit for bit the solo run, through
    two 64-step graph replays and an eager tail."""
    b = _batch(SMALL, "instances")
    lbm.lbm_batch_step(b, 131)
    lbm.lbm_batch_synchronize(b)
    assert lbm.lbm_batch_get_config(b)["mode"] == 2
    for i, s in enumerate(SMALL):
        p = _params(*s)
        solo = lbm.Simulation(p)
        solo.init_tgv(seed=5, noise_amp=0.02)
        solo.step(131)
        fs, gs = solo.populations()
        fb, gb = _pops(lbm.lbm_batch_instance(b, i), p)
        assert np.array_equal(fb, fs) and np.array_equal(gb, gs), i
        assert lbm.lbm_step_count(lbm.lbm_batch_instance(b, i)) == 131
        solo.close()
    # switching drivers mid-run keeps the state (the graph is rebuilt)
    lbm.lbm_batch_set_mode(b, "per_step")
    lbm.lbm_batch_step(b, 64)
    lbm.lbm_batch_set_mode(b, "instances")
    lbm.lbm_batch_step(b, 64)
    lbm.lbm_batch_synchronize(b)
    assert all(np.isfinite(d["Ek"]) and d["step"] == 259 for d in lbm.lbm_batch_diagnostics(b))
    lbm.lbm_batch_destroy(b)


def test_batch_instance_against_oracle():
    specs = [(16, "27x19", "sc", 100.0, 0.5), (12, "19x7", "guo", 80.0, 0.2)]
    b = _batch(specs, block=(16, 8))
    lbm.lbm_batch_step(b, 40)
    lbm.lbm_batch_synchronize(b)
    for i, s in enumerate(specs):
        p = _params(*s)
        o = oracle_for(p)
        o.init_fields(*I.tgv_fields(p.nx, 0.04, seed=5, noise_amp=0.02))
        o.step(40)
        qf, qg = lbm.PAIR_Q[p.pair]
        fb, gb = _pops(lbm.lbm_batch_instance(b, i), p)
        fo, go = o.populations()
        fo, go = fo[slot_map(qf)], go[slot_map(qg)]
        _, wf, _ = lbm.lbm_velocity_set(qf)
        assert np.max(np.abs(fb - fo)) <= 1e-5 * np.max(np.abs(fo - wf[:, None]))
        d = lbm.lbm_batch_diagnostics(b)[i]
        do = o.diagnostics()
        assert abs(d["Ek"] - do["Ek"]) / do["Ek"] < 1e-5
    lbm.lbm_batch_destroy(b)


def sweep_specs():
    """The 64-instance sweep: sizes {32, 48, 64, 96}^3 x Fr {1, 0.5, 0.2, 0.1}
    x forcing {Guo, Shan-Chen} x pair {D3Q19xD3Q7, D3Q27xD3Q19}, Re 200."""
    return [(n, pair, forcing, 200.0, fr) for n in (32, 48, 64, 96) for fr in (1.0, 0.5, 0.2, 0.1)
            for forcing in ("guo", "sc") for pair in ("19x7", "27x19")]


def test_sweep_64_instances_autotuned():
    specs = sweep_specs()
    assert len(specs) == 64
    b = _batch(specs, "persistent", 100)
    ms = lbm.lbm_batch_autotune(b, 2)
    assert ms > 0
    lbm.lbm_batch_step(b, 20)
    lbm.lbm_batch_synchronize(b)
    diags = lbm.lbm_batch_diagnostics(b)
    assert all(np.isfinite(d["Ek"]) and d["step"] == 20 for d in diags)
    # spot-check a few instances against solo runs with identical arithmetic
    for i in (0, 21, 42, 63):
        p = _params(*specs[i])
        solo = lbm.Simulation(p)
        solo.init_tgv(seed=5, noise_amp=0.02)
        solo.step(20)
        fs, _ = solo.populations()
        fb, _ = _pops(lbm.lbm_batch_instance(b, i), p)
        scale = np.max(np.abs(fs - lbm.lbm_velocity_set(lbm.PAIR_Q[p.pair][0])[1][:, None]))
        assert np.max(np.abs(fb - fs)) <= 1e-6 * scale, i
        solo.close()
    lbm.lbm_batch_destroy(b)


def test_barrier_timeout_returns_an_error_and_the_context_survives():
    b = _batch(SMALL, "persistent", 5)
    # every dependency wait expects one completion more than exists; each
    # wait gives up after 2000 polls
    lbm.lbm_batch_set_barrier_test(b, 1, 2000)
    lbm.lbm_batch_step(b, 5)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_batch_synchronize(b)
    assert ei.value.code == -4  # LBM_ETIMEOUT
    # back to normal: the device and the batch still work
    lbm.lbm_batch_set_barrier_test(b, 0, 1 << 22)
    lbm.lbm_batch_init_tgv(b, seed=5, noise_amp=0.02)
    lbm.lbm_batch_step(b, 12)
    lbm.lbm_batch_synchronize(b)
    assert all(np.isfinite(d["Ek"]) for d in lbm.lbm_batch_diagnostics(b))
    lbm.lbm_batch_destroy(b)


def test_batch_rejects_unsupported_instances():
    p = _params(16, "27x19", "guo", 100.0, 0.5)
    p.storage = 1
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_batch_create([p])
    assert ei.value.code == -6
