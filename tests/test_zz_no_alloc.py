"""The allocation-free diagnostics entry point against the regular one.

lbm_diagnostics_noalloc exists for callers that may not allocate device
memory themselves or let a library do it: programs that route every device
allocation through their own pool, code that cannot afford the device-wide
synchronisation that cudaMalloc/cudaFree imply while other streams are busy,
or a process that is out of headroom. Its scratch is a fixed array compiled
into the library, shared by every call, so this test calls it twice in a row
(with steps in between) and each time compares it with lbm_diagnostics on the
same state. The two sum the same FP32 per-node values over different thread
partitions (compensated FP32 within a thread, FP64 across threads): energies,
dissipation, mass and the maximum speed agree within 1e-10 relative; the total
momentum, a sum of O(1e-2) terms that cancels to O(1e-1), within 1e-6
absolute (5e-10 of the sum of |j| over the 48^3 nodes). This file is
collected last so that a failure here leaves every other test already run.
"""
import math

import pytest

from paper_2605_14505_gb300 import lbm

pytestmark = pytest.mark.gpu

KEYS = ("Ek", "Ep", "eps_k", "mass_f", "mass_g", "umax")


def _close(a, b, rel=1e-10, abs_=1e-12):
    return abs(a - b) <= rel * max(abs(a), abs(b)) + abs_


@pytest.mark.parametrize("pair", ["27x19", "19x7"])
@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_noalloc_diagnostics_match_two_calls_in_a_row(storage, pair):
    """FP32 and FP16 stores (the latter in the half-row order, read through the
    same node addressing), the D3Q27xD3Q19 pair and the D3Q19xD3Q7 pair (whose
    D3Q7 scalar set takes the diagnostics' explicit-equilibrium branch)."""
    n = 48
    p = lbm.lbm_params_from_physics(n, n, n, pair, "sc", 200.0, 0.2, 1.0, 0.04)
    sim = lbm.Simulation(p, storage=storage)
    sim.init_tgv(seed=11, noise_amp=0.01)
    for steps in (37, 13):  # odd layout first, then the natural layout
        sim.step(steps)
        ref = sim.diagnostics()
        got = lbm.lbm_diagnostics_noalloc(sim.h)
        assert got["step"] == ref["step"]
        for key in KEYS:
            assert _close(got[key], ref[key]), (key, got[key], ref[key])
        for key in ("mom_x", "mom_y", "mom_z"):
            assert _close(got[key], ref[key], abs_=1e-6), (key, got[key], ref[key])
        assert math.isnan(got["eps_p"]) and math.isnan(got["eps_k_curl"])
        assert got["t"] == ref["t"] and got["Ek_phys"] == pytest.approx(ref["Ek_phys"], rel=1e-10)
    sim.close()


def test_noalloc_diagnostics_small_lattice():
    """A lattice smaller than one block of nodes per SM: fewer blocks than the
    4-per-SM grid, none of them without nodes."""
    n = 8
    p = lbm.lbm_params_from_physics(n, n, n, "27x19", "guo", 100.0, 0.5, 1.0, 0.04)
    sim = lbm.Simulation(p)
    sim.init_tgv(seed=3, noise_amp=0.01)
    sim.step(5)
    ref = sim.diagnostics()
    got = lbm.lbm_diagnostics_noalloc(sim.h)
    for key in KEYS:
        assert _close(got[key], ref[key]), (key, got[key], ref[key])
    sim.close()


def test_noalloc_diagnostics_reject_lattices_beyond_the_scratch():
    # 520^3 nodes exceed the 512^3 capacity; the check comes before any device
    # work, so nothing is allocated for this handle
    p = lbm.lbm_params_from_physics(520, 520, 520, "19x7", "guo", 200.0, 0.2, 1.0, 0.04)
    h = lbm.lbm_create_params(p)
    try:
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_diagnostics_noalloc(h)
        assert ei.value.code == -1
        assert "static diagnostics scratch" in str(ei.value)
    finally:
        lbm.lbm_destroy(h)
