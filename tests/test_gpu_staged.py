"""The tile-staged step kernel (16-bit storage; rows brought into shared
memory by a producer warp's bulk asynchronous copies on mbarriers, two nodes
per consumer thread):
against the direct-load pair kernel, against the oracle, at the bench size by
sampling, and its bounded waits (made to run out on purpose with a test hook
that expects more bytes than the copies deliver: the kernel returns, the next
synchronize reports LBM_ETIMEOUT, the context stays usable)."""
import numpy as np
import pytest

import stgv_inputs as I
from paper_2605_14505_gb300 import lbm

from _helpers import gpu_sim, lattice_params, oracle_for, slot_map

pytestmark = pytest.mark.gpu

LAM = 2.0 ** -10


def _pair_sims(shape, pair, forcing, storage, seed=9):
    N = 3e-3
    p = lattice_params(*shape, pair, forcing, 0.55, 0.6, N * LAM, -N / LAM)
    n3 = shape[0] * shape[1] * shape[2]
    rho, u, rp = I.random_fields(*shape, seed, 0.05, 0.01, 0.02 / LAM)
    xf, xg = I.neq_noise(n3, seed + 1), I.neq_noise(n3, seed + 2)
    a = gpu_sim(p, storage)
    b = gpu_sim(p, storage)
    lbm.lbm_set_tile_staging(a.h, True)    # staged
    lbm.lbm_set_tile_staging(b.h, False)   # direct loads, two nodes per thread
    for s in (a, b):
        s.init_fields(rho, u, rp, xf, xg, 1e-3)
    return p, a, b


def _same_state(dst, src):
    """dst's store := src's store, byte for byte (any AA layout; both lattices
    have taken the same number of steps)."""
    import torch

    src.synchronize()
    dst.synchronize()
    dst._store.copy_(src._store)
    torch.cuda.synchronize()


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("pair,forcing", [("27x19", "sc"), ("27x19", "guo"), ("19x7", "edm"), ("19x7", "hcz")])
@pytest.mark.parametrize("shape,width", [((64, 3, 2), 64), ((128, 5, 3), 128), ((192, 2, 2), 64),
                                         ((256, 2, 3), 256), ((512, 1, 2), 256)])
def test_staged_matches_pair_kernel(storage, pair, forcing, shape, width):
    """Same per-node arithmetic and stores, only the loads differ. Before each
    step the staged lattice gets the direct-load lattice's store, so both
    kernels update the same state at each AA parity; the compiler may contract
    the FP32 arithmetic differently in the two kernels, so the results must
    agree to one storage ulp. Covers tiles of 64 to 256 nodes, several tiles
    per row and the x = 0 wrap of the odd step's copies."""
    p, a, b = _pair_sims(shape, pair, forcing, storage)
    assert lbm.lbm_uses_tile_staging(a.h) == width
    assert lbm.lbm_uses_tile_staging(b.h) == 0
    qf, qg = lbm.PAIR_Q[p.pair]
    _, wf, _ = lbm.lbm_velocity_set(qf)
    _, wg, _ = lbm.lbm_velocity_set(qg)
    ulp = 2.0 ** -10 if storage == "fp16" else 2.0 ** -7
    # FP32 rounding of the collision's O(1e-2) terms, which can leave a result
    # near zero a few 1e-9 apart (then more than one ulp of a BF16 value
    # there), and the FP16 subnormal spacing
    tiny = 2.0 ** -24
    for step in range(4):  # even, odd, even, odd
        _same_state(a, b)
        a.step(1)
        b.step(1)
        a.synchronize()
        fa, ga = a.populations()
        fb, gb = b.populations()
        # one ulp of the larger of the two stored deviations
        sf = np.maximum(np.abs(fa - wf[:, None]), np.abs(fb - wf[:, None]))
        sg = np.maximum(np.abs(ga - p.rho0 * wg[:, None]), np.abs(gb - p.rho0 * wg[:, None]))
        ef = np.abs(fa - fb) - (ulp * sf + tiny)
        eg = np.abs(ga - gb) - (ulp * sg + tiny)
        assert np.all(ef <= 1e-12), (step, float(np.max(ef)), int(np.sum(ef > 0)))
        assert np.all(eg <= 1e-12), (step, float(np.max(eg)), int(np.sum(eg > 0)))
    a.close()
    b.close()


@pytest.mark.parametrize("forcing", ["guo", "sc", "edm", "hcz"])
def test_staged_fp16_against_oracle(forcing):
    """FP16 storage through the staged kernel, one and two steps against the
    oracle started from the same (FP16-representable) populations."""
    N = 3e-3
    shape = (128, 6, 4)
    n3 = shape[0] * shape[1] * shape[2]
    p = lattice_params(*shape, "27x19", forcing, 0.53, 0.56, N * LAM, -N / LAM)
    g = gpu_sim(p, "fp16")
    lbm.lbm_set_tile_staging(g.h, True)
    rho, u, rp = I.random_fields(*shape, 3, 0.05, 0.01, 0.02 / LAM)
    g.init_fields(rho, u, rp, I.neq_noise(n3, 4), I.neq_noise(n3, 5), 1e-3)
    assert lbm.lbm_uses_tile_staging(g.h) == 128
    o = oracle_for(p)
    f0, g0 = g.populations()
    o.set_populations(f0[np.argsort(slot_map(27))], g0[np.argsort(slot_map(19))])
    _, wf, _ = lbm.lbm_velocity_set(27)
    _, wg, _ = lbm.lbm_velocity_set(19)
    for _ in range(2):
        g.step(1)
        o.step(1)
        fg, gg = g.populations()
        fo, go = o.populations()
        fo, go = fo[slot_map(27)], go[slot_map(19)]
        df, dg = fo - wf[:, None], go - p.rho0 * wg[:, None]
        assert np.max(np.abs(fg - fo)) <= 2.0 ** -10 * np.max(np.abs(df)) + 2.0 ** -23
        assert np.max(np.abs(gg - go)) <= 2.0 ** -10 * np.max(np.abs(dg)) + 2.0 ** -23
    g.close()


def test_staged_graph_replay_matches_eager():
    """The staged kernel inside the 64-step CUDA graph and launched eagerly
    give the same bits."""
    p = lbm.lbm_params_from_physics(64, 64, 64, "27x19", "sc", 100.0, 0.5, 1.0, 0.04)
    a = lbm.Simulation(p, storage="fp16")
    b = lbm.Simulation(p, storage="fp16")
    for s in (a, b):
        lbm.lbm_set_tile_staging(s.h, True)
    lbm.lbm_set_graphs(b.h, False)
    for s in (a, b):
        s.init_tgv(seed=3, noise_amp=1e-3)
        s.step(130)
        s.synchronize()
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    a.close()
    b.close()


def test_staged_wait_timeout_returns_an_error_and_the_context_survives():
    p = lbm.lbm_params_from_physics(64, 64, 64, "27x19", "sc", 100.0, 0.5, 1.0, 0.04)
    s = lbm.Simulation(p, storage="fp16")
    lbm.lbm_set_graphs(s.h, False)
    lbm.lbm_set_tile_staging(s.h, True)
    s.init_tgv(seed=1, noise_amp=1e-3)
    assert lbm.lbm_uses_tile_staging(s.h) == 64
    # each consumer warp also waits on a barrier that expects 16 bytes no copy
    # delivers; with 64 polls per wait even the waits on the real copies
    # usually run out first. Either way the consumers stop, the producer's
    # wait for the stages to come back runs out, and the producer waits for
    # its own copies (a fixed limit of its own) before the block returns.
    for spin in (64, 20000):
        lbm.lbm_set_stage_test(s.h, 16, spin)
        s.step(2)
        with pytest.raises(lbm.LbmError) as ei:
            s.synchronize()
        assert ei.value.code == -4  # LBM_ETIMEOUT
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_set_stage_test(s.h, 1 << 20, 64)
    assert ei.value.code == -1
    lbm.lbm_set_stage_test(s.h, 0, 1 << 22)
    s.init_tgv(seed=1, noise_amp=1e-3)
    s.step(4)
    s.synchronize()
    ref = lbm.Simulation(p, storage="fp16")
    lbm.lbm_set_tile_staging(ref.h, False)
    ref.init_tgv(seed=1, noise_amp=1e-3)
    ref.step(4)
    fa, _ = s.populations()
    fb, _ = ref.populations()
    _, wf, _ = lbm.lbm_velocity_set(27)
    assert np.all(np.abs(fa - fb) <= 2.0 ** -7 * np.abs(fb - wf[:, None]) + 1e-6)
    s.close()
    ref.close()
