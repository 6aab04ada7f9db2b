"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Populations are compared by velocity vector (the two sides use different slot
orders). Tolerances, FP32 storage: populations after one or two steps within
1e-5 of their deviation scale; after 1000 steps, E_k and E_p within 1e-5
relative (E_p relative to its maximum over the window) and velocity within
1e-4 U0 in L-infinity. FP16/BF16 deviation storage: E_k, E_p and eps_k within
1% of the FP64 trajectory.
"""
import numpy as np
import pytest

import stgv_inputs as I
from oracle import oracle as O
from paper_2605_14505_gb300 import lbm

from _helpers import gpu_sim, lattice_params, oracle_for, rel_err, slot_map

pytestmark = pytest.mark.gpu

LAM = 2.0 ** -10


def _random_pair(params, seed=5, amp=1e-3, u_amp=0.05, rp_amp=None):
    nx, ny, nz = params.nx, params.ny, params.nz
    n3 = nx * ny * nz
    if rp_amp is None:
        rp_amp = 0.02 / LAM
    rho, u, rp = I.random_fields(nx, ny, nz, seed, u_amp, 0.01, rp_amp)
    xf, xg = I.neq_noise(n3, seed + 1), I.neq_noise(n3, seed + 2)
    g = gpu_sim(params)
    g.init_fields(rho, u, rp, xf, xg, amp)
    o = oracle_for(params)
    o.init_fields(rho, u, rp, xf, xg, amp)
    return g, o


def _compare_pops(g, o, params, tol):
    qf, qg = lbm.PAIR_Q[params.pair]
    fg, gg = g.populations()
    fo, go = o.populations()
    pf, pg = slot_map(qf), slot_map(qg)
    _, wf, _ = lbm.lbm_velocity_set(qf)
    _, wg, _ = lbm.lbm_velocity_set(qg)
    fo, go = fo[pf], go[pg]
    sf = np.max(np.abs(fo - wf[:, None]))
    sg = np.max(np.abs(go - params.rho0 * wg[:, None]))
    ef = np.max(np.abs(fg - fo)) / sf
    eg = np.max(np.abs(gg - go)) / sg
    assert ef < tol and eg < tol, (ef, eg)
    return ef, eg


@pytest.mark.parametrize("pair", ["27x19", "19x7"])
@pytest.mark.parametrize("forcing", ["guo", "sc", "edm", "hcz"])
def test_population_parity_one_and_two_steps(pair, forcing):
    """One step leaves the AA store in its swapped layout, two in the natural
    one; both must read back as the oracle's populations. 40 x 12 x 6 spans two
    32-wide tiles in x with a ragged tail and a ragged tile in y."""
    N = 3e-3
    p = lattice_params(40, 12, 6, pair, forcing, 0.53, 0.56, N * LAM, -N / LAM)
    g, o = _random_pair(p)
    _compare_pops(g, o, p, 1e-5)
    for _ in range(2):
        g.step(1)
        o.step(1)
        _compare_pops(g, o, p, 1e-5)


@pytest.mark.parametrize("scalar_mode,sc_shift", [(1, 1.0), (0, 0.5)])
def test_population_parity_reading_flags(scalar_mode, sc_shift):
    """The Chai-Shi scalar pair and the Shan-Chen shift exactly as printed in Eq. 10."""
    N = 3e-3
    p = lattice_params(33, 7, 5, "27x19", "sc", 0.55, 0.7, N * LAM, -N / LAM, scalar_mode=scalar_mode,
                       sc_shift=sc_shift)
    g, o = _random_pair(p)
    for _ in range(3):
        g.step(1)
        o.step(1)
    _compare_pops(g, o, p, 1e-5)


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 1), (1, 1, 5), (33, 5, 3), (64, 2, 2)])
def test_degenerate_and_ragged_shapes(shape):
    """Single-node and thin periodic lattices (x - 1 wraps onto x itself) and a
    ragged 33-wide row, 4 steps, against the oracle."""
    N = 3e-3
    p = lattice_params(*shape, "27x19", "guo", 0.6, 0.6, N * LAM, -N / LAM)
    g, o = _random_pair(p)
    g.step(4)
    o.step(4)
    _compare_pops(g, o, p, 2e-5)


def test_zero_steps_and_call_order():
    p = lattice_params(8, 8, 8, "27x19", "guo", 0.6, 0.6, 1e-5, -4.0)
    g = gpu_sim(p)
    with pytest.raises(lbm.LbmError) as ei:
        g.step(1)
    assert ei.value.code == -7  # LBM_ESTATE: step before init
    with pytest.raises(lbm.LbmError) as ei:
        g.diagnostics()
    assert ei.value.code == -7
    g.init_tgv(0, 0.0)
    f0, _ = g.populations()
    g.step(0)
    f1, _ = g.populations()
    assert np.array_equal(f0, f1)
    with pytest.raises(lbm.LbmError):
        g.step(-1)


def test_invalid_parameters_rejected():
    p = lattice_params(8, 8, 8, "27x19", "guo", 0.5, 0.6, 1e-5, -4.0)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create_params(p)
    assert ei.value.code == -1
    p = lattice_params(8, 8, 4, "27x19", "guo", 0.6, 0.6, 1e-5, -4.0)
    g = gpu_sim(p)
    with pytest.raises(lbm.LbmError) as ei:
        g.init_tgv(0, 0.0)  # the Taylor-Green box is cubic
    assert ei.value.code == -1


def _run_both(n, pair, forcing, Re, Fr, steps, storage="fp32", every=None, U0=0.04):
    p = lbm.lbm_params_from_physics(n, n, n, pair, forcing, Re, Fr, 1.0, U0)
    g = gpu_sim(p, storage)
    o = oracle_for(p)
    rho, u, rp = I.tgv_fields(n, U0)
    g.init_fields(rho, u, rp)
    o.init_fields(rho, u, rp)
    every = every or steps
    series = []
    for _ in range(steps // every):
        g.step(every)
        o.step(every)
        series.append((g.diagnostics(), o.diagnostics()))
    return p, g, o, series


@pytest.mark.parametrize("pair,forcing", [("27x19", "sc"), ("27x19", "guo"), ("19x7", "edm")])
def test_fp32_1000_steps_tolerances(pair, forcing):
    """FP32 storage after 1000 steps of the 32^3 stratified TGV (Re 100, Fr 0.5):
    E_k, E_p relative error <= 1e-5 and velocity L-inf <= 1e-4 U0."""
    U0 = 0.04
    p, g, o, series = _run_both(32, pair, forcing, 100.0, 0.5, 1000, every=100, U0=U0)
    ep_max = max(s[1]["Ep"] for s in series)
    for dg, do in series:
        assert abs(dg["Ek"] - do["Ek"]) / do["Ek"] <= 1e-5, (dg["Ek"], do["Ek"])
        assert abs(dg["Ep"] - do["Ep"]) / ep_max <= 1e-5, (dg["Ep"], do["Ep"])
    _, ug, rg = g.fields()
    _, uo, ro = o.fields()
    assert np.max(np.abs(ug - uo)) <= 1e-4 * U0
    assert rel_err(rg, ro) < 1e-4


def test_c0_diagnostics_series():
    """The 32^3, D3Q27xD3Q19, Guo, Re 100, Fr 0.5 workload for its full 200
    steps, diagnostics every 50 steps, all estimators against the oracle."""
    p, g, o, series = _run_both(32, "27x19", "guo", 100.0, 0.5, 200, every=50)
    for dg, do in series:
        for key in ("Ek", "eps_k", "eps_k_curl"):
            assert abs(dg[key] - do[key]) / abs(do[key]) < 2e-5, (key, dg[key], do[key])
        for key in ("Ep", "eps_p"):
            assert abs(dg[key] - do[key]) / abs(do[key]) < 2e-4, (key, dg[key], do[key])
        # FP32 storage rounds each deviation every step: the totals random-walk
        # by ~1e-8 per node over this window (the oracle conserves to 1e-16)
        n3 = 32 ** 3
        assert abs(dg["mass_f"] - do["mass_f"]) / n3 < 1e-8
        assert abs(dg["mass_g"] - do["mass_g"]) / n3 < 1e-6
        # total momentum (~0 by symmetry) drifts by FP32 random-walk rounding only:
        # ~2e-9 per node per step over 32^3 nodes and 200 steps is ~6e-6
        for key in ("mom_x", "mom_y", "mom_z"):
            assert abs(dg[key] - do[key]) < 5e-5
        # the paper-unit block (Section 2.4: U = L = 1) from the handle's U0, L
        U0, L = p.U0, p.L
        assert abs(dg["t"] - do["step"] * U0 / L) < 1e-15 * (1 + dg["t"])
        for key in ("Ek", "Ep"):
            assert dg[key + "_phys"] == pytest.approx(dg[key] / U0 ** 2, rel=1e-15)
        for key in ("eps_k", "eps_p", "eps_k_curl"):
            assert dg[key + "_phys"] == pytest.approx(dg[key] * L / U0 ** 3, rel=1e-15)


@pytest.mark.parametrize("storage,tol", [("fp16", 0.01), ("bf16", 0.05)])
def test_reduced_precision_storage_error(storage, tol):
    """FP16/BF16 deviation storage with FP32 arithmetic: E_k, E_p, eps_k within
    `tol` of the FP64 oracle over 1000 steps of the 32^3 SC case (the precision
    target's 1 % for FP16; BF16 keeps 8 mantissa bits and is reported at 5 %)."""
    p, g, o, series = _run_both(32, "27x19", "sc", 100.0, 0.5, 1000, storage=storage, every=100)
    ep_max = max(s[1]["Ep"] for s in series)
    for dg, do in series:
        assert abs(dg["Ek"] - do["Ek"]) / do["Ek"] < tol, ("Ek", dg["Ek"], do["Ek"])
        assert abs(dg["Ep"] - do["Ep"]) / ep_max < tol, ("Ep", dg["Ep"], do["Ep"])
        assert abs(dg["eps_k"] - do["eps_k"]) / do["eps_k"] < tol, ("eps_k", dg["eps_k"], do["eps_k"])


def test_device_tgv_init_matches_host_generator():
    """lbm_init_tgv (Eq. 20 + SplitMix64 noise on the device) equals
    lbm_init_fields fed by the seeded host generator."""
    n, U0 = 24, 0.04
    p = lbm.lbm_params_from_physics(n, n, n, "27x19", "sc", 100.0, 0.5, 1.0, U0)
    a = gpu_sim(p)
    a.init_tgv(seed=1234, noise_amp=0.05)
    b = gpu_sim(p)
    b.init_fields(*I.tgv_fields(n, U0, seed=1234, noise_amp=0.05))
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.max(np.abs(fa - fb)) < 1e-9
    assert np.max(np.abs(ga - gb)) < 1e-9


def test_graph_replay_is_bitwise_eager():
    n = 48
    p = lbm.lbm_params_from_physics(n, n, n, "27x19", "sc", 200.0, 0.2, 1.0, 0.04)
    a = gpu_sim(p)
    b = gpu_sim(p)
    lbm.lbm_set_graphs(b.h, False)
    for s in (a, b):
        s.init_tgv(seed=3, noise_amp=0.01)
        s.step(129)  # 2 graph replays of 64 steps + 1 eager step for a
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_autotune_keeps_state_and_results():
    n = 40
    p = lbm.lbm_params_from_physics(n, n, n, "19x7", "guo", 200.0, 0.2, 1.0, 0.04)
    a = gpu_sim(p)
    b = gpu_sim(p)
    for s in (a, b):
        s.init_tgv(seed=9, noise_amp=0.01)
        s.step(3)
    f0, g0 = a.populations()
    ms = lbm.lbm_autotune(a.h, 2)
    assert ms > 0
    f1, g1 = a.populations()
    assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    assert a.step_count == 3
    a.step(10)
    b.step(10)  # block shape does not change the per-node arithmetic
    assert np.array_equal(a.populations()[0], b.populations()[0])


def test_per_parity_launch_shapes_give_the_same_bits():
    """FP16 D3Q27xD3Q19 at nx = 256 launches its even steps in 64 x 2 blocks
    and its odd steps as one row of 128 threads; the launch shape does not
    change the per-node arithmetic, so a lattice run with 64 x 2 on both
    parities gives the same bits, through both AA parities and the row-wrap
    lanes; the per-parity autotuner keeps the state."""
    shape = (256, 8, 4)
    N = 3e-3
    p = lattice_params(*shape, "27x19", "sc", 0.53, 0.56, N * LAM, -N / LAM)
    rho, u, rp = I.random_fields(*shape, 21, 0.05, 0.01, 0.02 / LAM)
    a = gpu_sim(p, "fp16")
    b = gpu_sim(p, "fp16")
    lbm.lbm_set_block(b.h, 64, 2)
    assert lbm.lbm_get_block(a.h) == (64, 2)
    for s in (a, b):
        s.init_fields(rho, u, rp)
        s.step(5)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    ms = lbm.lbm_autotune(a.h, 2)
    assert ms > 0
    f1, g1 = a.populations()
    assert np.array_equal(fa, f1) and np.array_equal(ga, g1) and a.step_count == 5
    for s in (a, b):
        s.step(4)
    assert np.array_equal(a.populations()[0], b.populations()[0])
    a.close()
    b.close()


def test_checkpoint_roundtrip():
    n = 16
    p = lbm.lbm_params_from_physics(n, n, n, "27x19", "edm", 100.0, 0.3, 1.0, 0.04)
    a = gpu_sim(p)
    a.init_tgv(seed=2, noise_amp=0.02)
    a.step(7)
    f, g = a.populations()
    b = gpu_sim(p)
    b.set_populations(f, g)
    a.step(5)
    b.step(5)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.max(np.abs(fa - fb)) == 0.0 and np.max(np.abs(ga - gb)) == 0.0


@pytest.mark.parametrize("mode", ["all", "even"])
@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("shape", [(2, 3, 2), (34, 6, 4), (64, 5, 3), (258, 2, 2)])
def test_pair_kernel_matches_single_node_kernel(mode, storage, shape):
    """16-bit storage with even nx runs two nodes per thread (on every step,
    or on even steps only); the per-node arithmetic is the one-node kernel's,
    so both agree to the storage rounding (nx = 2 makes x0 - 1 and x0 + 2
    wrap onto the pair itself)."""
    N = 3e-3
    p = lattice_params(*shape, "27x19", "sc", 0.55, 0.6, N * LAM, -N / LAM)
    n3 = shape[0] * shape[1] * shape[2]
    rho, u, rp = I.random_fields(*shape, 9, 0.05, 0.01, 0.02 / LAM)
    xf, xg = I.neq_noise(n3, 10), I.neq_noise(n3, 11)
    a = gpu_sim(p, storage)
    b = gpu_sim(p, storage)
    for s in (a, b):
        lbm.lbm_set_tile_staging(s.h, False)
    lbm.lbm_set_pairing(a.h, mode)
    lbm.lbm_set_pairing(b.h, "off")
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_pairing(b.h, 3)
    for s in (a, b):
        s.init_fields(rho, u, rp, xf, xg, 1e-3)
    for _ in range(3):  # odd, even, odd layouts
        a.step(1)
        b.step(1)
        fa, ga = a.populations()
        fb, gb = b.populations()
        _, wf, _ = lbm.lbm_velocity_set(27)
        rel = 2.0 ** -9 if storage == "fp16" else 2.0 ** -6
        assert np.all(np.abs(fa - fb) <= rel * np.abs(fb - wf[:, None]) + 1e-7)
        assert np.all(np.abs(ga - gb) <= rel * np.abs(gb) + 1e-7)


@pytest.mark.parametrize("forcing", ["guo", "sc", "edm", "hcz"])
def test_fp16_pair_kernel_against_oracle(forcing):
    """FP16 deviation storage, pair kernel, one and two steps against the
    oracle started from the same (FP16-representable) populations."""
    N = 3e-3
    p = lattice_params(40, 12, 6, "27x19", forcing, 0.53, 0.56, N * LAM, -N / LAM)
    g = gpu_sim(p, "fp16")
    rho, u, rp = I.random_fields(40, 12, 6, 3, 0.05, 0.01, 0.02 / LAM)
    g.init_fields(rho, u, rp, I.neq_noise(40 * 12 * 6, 4), I.neq_noise(40 * 12 * 6, 5), 1e-3)
    o = oracle_for(p)
    f0, g0 = g.populations()   # exactly what the GPU holds
    o.set_populations(f0[np.argsort(slot_map(27))], g0[np.argsort(slot_map(19))])
    for _ in range(2):
        g.step(1)
        o.step(1)
        fg, gg = g.populations()
        fo, go = o.populations()
        fo, go = fo[slot_map(27)], go[slot_map(19)]
        _, wf, _ = lbm.lbm_velocity_set(27)
        _, wg, _ = lbm.lbm_velocity_set(19)
        df, dg = fo - wf[:, None], go - p.rho0 * wg[:, None]
        # FP16 storage rounding (half an ulp, relative 2^-11, per step; the first
        # step's rounding is mixed into other slots by the second), plus FP32
        # arithmetic and the FP16 subnormal spacing
        assert np.max(np.abs(fg - fo)) <= 2.0 ** -10 * np.max(np.abs(df)) + 2.0 ** -23
        assert np.max(np.abs(gg - go)) <= 2.0 ** -10 * np.max(np.abs(dg)) + 2.0 ** -23


@pytest.mark.parametrize("pair", ["27x27", "19x19", "19x15", "15x7", "7x27"])
@pytest.mark.parametrize("forcing", ["guo", "sc"])
def test_other_stencil_pairs(pair, forcing):
    """The paper's other stencil pairs (Sections 3.2-3.3), FP32 storage: one and
    two steps against the oracle, and the diagnostics of the result."""
    N = 3e-3
    p = lattice_params(36, 10, 6, pair, forcing, 0.56, 0.58, N * LAM, -N / LAM)
    g, o = _random_pair(p, seed=13)
    for _ in range(2):
        g.step(1)
        o.step(1)
        _compare_pops(g, o, p, 1e-5)
    dg, do = g.diagnostics(), o.diagnostics()
    for key in ("Ek", "Ep", "eps_k", "eps_p", "eps_k_curl"):
        assert abs(dg[key] - do[key]) <= 2e-5 * abs(do[key]) + 1e-14, (key, dg[key], do[key])


@pytest.mark.parametrize("pair", ["27x27", "19x19", "19x15", "15x7", "7x27"])
@pytest.mark.parametrize("forcing", ["guo", "sc"])
def test_other_stencil_pairs_fp16(pair, forcing):
    """The paper's other stencil pairs with FP16 deviation storage (pair
    kernel, even nx): one and two steps against the oracle started from the
    same FP16-representable populations, within the storage rounding."""
    N = 3e-3
    nx, ny, nz = 36, 10, 6
    p = lattice_params(nx, ny, nz, pair, forcing, 0.56, 0.58, N * LAM, -N / LAM)
    qf, qg = lbm.PAIR_Q[p.pair]
    g = gpu_sim(p, "fp16")
    n3 = nx * ny * nz
    rho, u, rp = I.random_fields(nx, ny, nz, 17, 0.05, 0.01, 0.02 / LAM)
    g.init_fields(rho, u, rp, I.neq_noise(n3, 18), I.neq_noise(n3, 19), 1e-3)
    o = oracle_for(p)
    f0, g0 = g.populations()
    o.set_populations(f0[np.argsort(slot_map(qf))], g0[np.argsort(slot_map(qg))])
    _, wf, _ = lbm.lbm_velocity_set(qf)
    _, wg, _ = lbm.lbm_velocity_set(qg)
    for _ in range(2):
        g.step(1)
        o.step(1)
        fg, gg = g.populations()
        fo, go = o.populations()
        fo, go = fo[slot_map(qf)], go[slot_map(qg)]
        df, dg = fo - wf[:, None], go - p.rho0 * wg[:, None]
        assert np.max(np.abs(fg - fo)) <= 2.0 ** -10 * np.max(np.abs(df)) + 2.0 ** -23, pair
        assert np.max(np.abs(gg - go)) <= 2.0 ** -10 * np.max(np.abs(dg)) + 2.0 ** -23, pair


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("shape", [(1, 1, 1), (33, 5, 3), (7, 2, 9)])
def test_16bit_odd_nx_one_node_kernel_against_oracle(storage, shape):
    """Odd nx (no pairs) runs the one-node 16-bit kernel: two steps against the
    oracle from the same 16-bit-representable populations, within two storage
    roundings of the node scale (one per step)."""
    N = 3e-3
    p = lattice_params(*shape, "27x19", "sc", 0.53, 0.56, N * LAM, -N / LAM)
    n3 = shape[0] * shape[1] * shape[2]
    g = gpu_sim(p, storage)
    rho, u, rp = I.random_fields(*shape, 21, 0.05, 0.01, 0.02 / LAM)
    g.init_fields(rho, u, rp, I.neq_noise(n3, 22), I.neq_noise(n3, 23), 1e-3)
    o = oracle_for(p)
    f0, g0 = g.populations()
    o.set_populations(f0[np.argsort(slot_map(27))], g0[np.argsort(slot_map(19))])
    ulp = 2.0 ** -11 if storage == "fp16" else 2.0 ** -8
    _, wf, _ = lbm.lbm_velocity_set(27)
    _, wg, _ = lbm.lbm_velocity_set(19)
    for _ in range(2):
        g.step(1)
        o.step(1)
        fg, gg = g.populations()
        fo, go = o.populations()
        fo, go = fo[slot_map(27)], go[slot_map(19)]
        df, dg = fo - wf[:, None], go - p.rho0 * wg[:, None]
        assert np.max(np.abs(fg - fo)) <= 4 * ulp * np.max(np.abs(df)) + 2.0 ** -23
        assert np.max(np.abs(gg - go)) <= 4 * ulp * np.max(np.abs(dg)) + 2.0 ** -23


@pytest.mark.parametrize("storage,n,staging", [("fp32", 40, False), ("fp16", 40, False), ("fp16", 33, False),
                                               ("bf16", 64, True)])
@pytest.mark.parametrize("pair", ["27x19", "19x7"])
def test_fused_step_diagnostics_match_separate_calls(storage, n, staging, pair):
    """lbm_step_diagnostics (diagnostics reduced inside the first step) equals
    lbm_diagnostics followed by lbm_step on the same state. FP32 storage: the
    same FP32 node values summed per step-kernel block instead of per
    diagnostics block, so within 1e-9 relative; 16-bit storage: the node
    moments come from the step's short-form FP32 arithmetic, so within 1e-6.
    The momentum totals cancel: with 16-bit storage each node's FP32 momentum
    (|j| <~ 0.05) differs between the short and the exact forms by a few FP32
    ulps, and those differences add up like a random walk over the n^3 nodes,
    so the bound is 4 * sqrt(n^3) * 0.05 * 4 * 2^-24 absolute (9e-6 at 33^3,
    1.2e-5 at 40^3); with FP32 storage (the same arithmetic) 1e-6.
    The state afterwards is within
    FP32 rounding of the plain steps, at both AA parities. Covers the one-node
    (odd n) and two-node 16-bit kernels, and tile staging switched on (the
    diagnosing step then runs the two-node kernel, the others the staged one)."""
    p = lbm.lbm_params_from_physics(n, n, n, pair, "sc", 200.0, 0.2, 1.0, 0.04)
    a = gpu_sim(p, storage)
    b = gpu_sim(p, storage)
    if staging:
        for s in (a, b):
            lbm.lbm_set_tile_staging(s.h, True)
    for s in (a, b):
        s.init_tgv(seed=5, noise_amp=0.01)
        s.step(3)   # odd layout
    for chunk in (7, 12):
        da = a.step_diagnostics(chunk)
        db = b.diagnostics()
        b.step(chunk)
        assert da["step"] == db["step"]
        rel = 1e-9 if storage == "fp32" else 1e-6
        for key in ("Ek", "Ep", "eps_k", "eps_p", "eps_k_curl", "mass_f", "mass_g", "umax"):
            assert abs(da[key] - db[key]) <= rel * abs(db[key]) + 1e-15, (key, da[key], db[key])
        mom_tol = 1e-6 if storage == "fp32" else 4 * np.sqrt(float(n) ** 3) * 0.05 * 4 * 2.0 ** -24
        for key in ("mom_x", "mom_y", "mom_z"):
            assert abs(da[key] - db[key]) <= mom_tol, (key, da[key], db[key], mom_tol)
        a.synchronize()
        fa, ga = a.populations()
        fb, gb = b.populations()
        qf, _ = lbm.PAIR_Q[p.pair]
        _, wf, _ = lbm.lbm_velocity_set(qf)
        tol = {"fp32": 1e-6, "fp16": 2.0 ** -9, "bf16": 2.0 ** -6}[storage]
        assert np.all(np.abs(fa - fb) <= tol * np.max(np.abs(fb - wf[:, None])) + 1e-12)
        assert np.all(np.abs(ga - gb) <= tol * np.max(np.abs(gb)) + 1e-12)
    with pytest.raises(lbm.LbmError):
        a.step_diagnostics(0)


def test_prefetched_initialisation_matches_init_fields():
    """lbm_prefetch_fields + lbm_init_prefetched (copies on a side stream,
    overlapping the running steps, two alternating buffers) give the same
    populations as lbm_init_fields, bit for bit, over three rounds; misuse is
    reported."""
    n = 24
    p = lbm.lbm_params_from_physics(n, n, n, "27x19", "sc", 100.0, 0.5, 1.0, 0.04)
    a = gpu_sim(p)
    b = gpu_sim(p)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_init_prefetched(a.h)
    fields = [I.tgv_fields(n, 0.04, seed=s, noise_amp=0.05) for s in (1, 2, 3)]
    lbm.lbm_prefetch_fields(a.h, *fields[0])
    with pytest.raises(lbm.LbmError):
        lbm.lbm_prefetch_fields(a.h, *fields[0])
    for k in range(3):
        lbm.lbm_init_prefetched(a.h)
        if k + 1 < 3:
            lbm.lbm_prefetch_fields(a.h, *fields[k + 1])
        a.step(5)
        b.init_fields(*fields[k])
        b.step(5)
        a.synchronize()
        fa, ga = a.populations()
        fb, gb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), k
        assert a.step_count == 5


@pytest.mark.parametrize("storage,nx", [("fp16", 6), ("bf16", 8), ("fp16", 5), ("fp32", 6), ("bf16", 2)])
def test_store_row_order(storage, nx):
    """The store's element order, which lbm_attach exposes: slot-major, then z,
    y, and within a row node x at position x (FP32 storage, odd nx) or, for
    16-bit storage with even nx, the half-row order: position 2 x for
    x < nx / 2, 2 (x - nx / 2) + 1 above, so that 32-bit word k holds nodes k
    and k + nx / 2."""
    import torch

    ny, nz = 3, 2
    p = lattice_params(nx, ny, nz, "27x19", "sc", 0.55, 0.6, 3e-3 * LAM, -3e-3 / LAM)
    n3 = nx * ny * nz
    qf, qg = 27, 19
    _, wf, _ = lbm.lbm_velocity_set(qf)
    _, wg, _ = lbm.lbm_velocity_set(qg)
    # deviations that name their slot and node, exact in every storage type:
    # multiples of 2^-12 below 2^-4 (8 significant bits at most)
    code_f = ((np.arange(qf)[:, None] * 7 + np.arange(n3)[None, :] * 3) % 253 + 1) * 2.0 ** -12
    code_g = -((np.arange(qg)[:, None] * 5 + np.arange(n3)[None, :] * 11) % 251 + 1) * 2.0 ** -12
    s = gpu_sim(p, storage)
    s.set_populations(wf[:, None] + code_f, p.rho0 * wg[:, None] + code_g)
    s.synchronize()
    dt = {"fp32": torch.float32, "fp16": torch.float16, "bf16": torch.bfloat16}[storage]
    raw = s._store.view(dt).double().cpu().numpy()
    rf = raw[: qf * n3].reshape(qf, n3)
    rg = raw[qf * n3: (qf + qg) * n3].reshape(qg, n3)
    half = nx // 2 if (storage != "fp32" and nx % 2 == 0) else 0
    x = np.arange(n3) % nx
    pos = x if half == 0 else np.where(x < half, 2 * x, 2 * (x - half) + 1)
    elem = np.arange(n3) - x + pos
    assert np.array_equal(np.sort(elem), np.arange(n3))
    assert np.array_equal(rf[:, elem], code_f)
    assert np.array_equal(rg[:, elem], code_g)
    # and the library reads its own order back (w + code - w: one FP64 rounding)
    f, g = s.populations()
    assert np.max(np.abs(f - wf[:, None] - code_f)) < 1e-12
    assert np.max(np.abs(g - p.rho0 * wg[:, None] - code_g)) < 1e-12
    s.close()


def test_field_initialisation_rounds_fp64_fields_to_nearest_even():
    """lbm_init_fields rounds the FP64 host fields to FP32 as IEEE 754 does
    (to nearest, ties to even) before the FP32 equilibria. With u = 0 the
    rest slots hold w_0 float(rho - 1) and w_0^g (float(rho') + 0); with rho = 1 and
    u = (u_x, 0, 0) the f rest slot holds w_0 (-(3/2) float(u_x)^2). Fed
    random values, exact ties between adjacent floats (both parities of the
    lower one), values that round up into the next binade, float-subnormal
    and double-subnormal values and zeros of both signs, the FP32 store must
    equal numpy's float32 rounding bit for bit."""
    import torch

    rng = np.random.default_rng(3)
    anchors = rng.uniform(-0.3, 0.3, 400).astype(np.float32)
    nxt = np.nextafter(anchors, np.float32(np.inf))
    ties = (anchors.astype(np.float64) + nxt.astype(np.float64)) / 2.0
    rand = rng.uniform(-1.0, 1.0, 400) * 10.0 ** rng.integers(-30, 3, 400).astype(np.float64)
    up = np.ldexp(2.0 - 2.0 ** -30, rng.integers(-40, -2, 100)) * rng.choice([-1.0, 1.0], 100)
    tiny = np.array([1e-40, -3e-42, 5e-324, -2.5e-310, 1e-45, 7e-46, 1.4e-45, 0.0, -0.0])
    vals = np.concatenate([ties, rand, up, tiny])
    nx, ny, nz = 64, 16, 4
    n3 = nx * ny * nz
    k = len(vals)
    assert 3 * k <= n3
    rho = np.ones(n3)
    u = np.zeros(3 * n3)
    rp = np.zeros(n3)
    # rho - 1 path: ties and values in the range where 1 + t is exact
    drho = np.concatenate([ties, rng.uniform(-0.3, 0.3, k - len(ties))])
    rho[:k] = 1.0 + drho
    # u_x path: values whose FP32 square stays normal (a square that underflows
    # to zero says nothing about the conversion)
    rand_u = np.where(np.abs(rand) < 1e-18, 0.1, rand)
    u[k:2 * k] = np.concatenate([ties, rand_u, up, np.full(len(tiny), 0.25)])
    rp[2 * k:3 * k] = vals
    p = lattice_params(nx, ny, nz, "27x19", "sc", 0.55, 0.6, 0.0, 0.0)
    s = gpu_sim(p, "fp32")
    s.init_fields(rho, u, rp)
    s.synchronize()
    raw = s._store.view(torch.float32).cpu().numpy()
    f0, g0 = raw[:n3], raw[27 * n3: 28 * n3]   # rest slots (slot 0 of f and of g)
    w0 = np.float32(8.0 / 27.0)
    w0g = np.float32(1.0 / 3.0)
    with np.errstate(over="ignore", under="ignore"):
        exp_rho = w0 * (rho[:k] - 1.0).astype(np.float32)
        uxf = u[k:2 * k].astype(np.float32)
        exp_u = w0 * (np.float32(-1.5) * (uxf * uxf))
        # the FMA adds the (zero) equilibrium term: -0 + 0 = +0, as IEEE rounds
        exp_rp = w0g * (rp[2 * k:3 * k].astype(np.float32) + np.float32(0.0))
    assert np.array_equal(f0[:k].view(np.uint32), exp_rho.view(np.uint32))
    assert np.array_equal(f0[k:2 * k].view(np.uint32), exp_u.view(np.uint32))
    assert np.array_equal(g0[2 * k:3 * k].view(np.uint32), exp_rp.view(np.uint32))
    s.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_device_fields_equal_host_fields(storage):
    """lbm_get_fields_device writes the same FP64 fields as lbm_get_fields
    (after an odd step count, so the swapped AA arrangement is read)."""
    import torch

    n = 24
    p = lbm.lbm_params_from_physics(n, n, n, "27x19", "sc", 100.0, 0.5, 1.0, 0.04)
    s = gpu_sim(p, storage)
    s.init_tgv(seed=3, noise_amp=0.01)
    s.step(7)
    rho, u, rp = s.fields()
    drho, du, drp = s.fields_device()
    assert np.array_equal(drho.cpu().numpy(), rho)
    assert np.array_equal(du.cpu().numpy(), u)
    assert np.array_equal(drp.cpu().numpy(), rp)
    # one output only; a host pointer is rejected
    only_u = torch.zeros((3, n ** 3), dtype=torch.float64, device="cuda")
    lbm.lbm_get_fields_device(s.h, None, only_u.data_ptr(), None)
    s.synchronize()
    assert np.array_equal(only_u.cpu().numpy(), u)
    host = np.zeros(n ** 3)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_get_fields_device(s.h, host.ctypes.data, None, None)
    assert ei.value.code == -1
    s.close()


def test_gpu_spectrum_matches_host_spectrum():
    """The cuFFT spectrum of the device field equals the numpy one."""
    from paper_2605_14505_gb300 import post

    n = 32
    p = lbm.lbm_params_from_physics(n, n, n, "27x19", "sc", 400.0, 1.0, 0.7, 0.0577)
    s = gpu_sim(p)
    s.init_tgv(seed=1, noise_amp=0.01)
    s.step(50)
    _, u, _ = s.fields()
    _, du, _ = s.fields_device()
    k1, E1 = post.energy_spectrum(u, n)
    k2, E2 = post.energy_spectrum_device(du, n)
    assert np.array_equal(k1, k2)
    assert np.allclose(E1, E2, rtol=1e-10, atol=1e-22)
    s.close()


def test_nonfinite_state_is_reported():
    """A NaN population (set on the host; NaN arithmetic does not fault) makes
    every diagnostics entry point return LBM_ENONFINITE, with the record still
    filled; the state and the context stay usable (re-initialised)."""
    p = lattice_params(16, 8, 4, "27x19", "guo", 0.6, 0.6, 1e-5, -4.0)
    s = gpu_sim(p)
    rho, u, rp = I.random_fields(16, 8, 4, 21, 0.03, 0.01, 0.1)
    s.init_fields(rho, u, rp)
    f, g = s.populations()
    f[3, 17] = np.nan
    s.set_populations(f, g)
    with pytest.raises(lbm.LbmError) as ei:
        s.diagnostics()
    assert ei.value.code == -5
    d = s.diagnostics(allow_nonfinite=True)
    assert not np.isfinite(d["mass_f"]) and d["step"] == 0
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_diagnostics_noalloc(s.h)
    assert ei.value.code == -5
    with pytest.raises(lbm.LbmError) as ei:
        s.step_diagnostics(2)
    assert ei.value.code == -5
    s.init_fields(rho, u, rp)
    s.step(3)
    assert np.isfinite(s.diagnostics()["Ek"])
    s.close()
