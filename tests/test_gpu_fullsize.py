"""Parity at the workloads' full sizes, in the launch configuration the bench
uses (default block shape, CUDA-graph replay on), by sampling.

For sampled nodes x the CUDA path's populations f(x, t) are read back
(lbm_sample_populations); the oracle collides exactly those values on a 1^3
periodic lattice, where streaming is the identity, giving f*(x); the CUDA
path's f_i(x + e_i, t + 1) must equal f*_i(x). This checks every slot of the
stream-and-collide update at both AA parities, at any lattice size, against
the FP64 oracle. Tolerances: FP32 storage 2e-6 of the node's deviation scale
(one step of FP32 arithmetic); FP16/BF16 storage the storage rounding of the
output, 2^-10 / 2^-7 of each value's deviation plus 2e-6 of the scale, plus
2^-24 for FP16 (the absolute spacing of its subnormal range).
Invariants checked at the same sizes: total mass is conserved and the total
lattice momentum gains exactly sum_x F per step, up to FP32 rounding.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_14505_gb300 import lbm

from _helpers import slot_map

pytestmark = pytest.mark.gpu


def _sample_nodes(n, count, seed):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, n ** 3, size=count)
    corners = [0, n - 1, n * n - 1, n ** 3 - 1, n ** 3 - n, (n // 2) * (n * n + n + 1)]
    return np.unique(np.concatenate([idx, corners]).astype(np.int64))


def _neighbor(n, node, e):
    x = node % n
    y = (node // n) % n
    z = node // (n * n)
    return ((x + e[0]) % n) + n * (((y + e[1]) % n) + n * ((z + e[2]) % n))


def _check_one_step(sim, p, nodes, rel_store, abs_store):
    """Sample f(x, t), step once, compare f_i(x + e_i, t + 1) with the oracle."""
    qf, qg = lbm.PAIR_Q[p.pair]
    ef, wf, _ = lbm.lbm_velocity_set(qf)
    eg, wg, _ = lbm.lbm_velocity_set(qg)
    f0, g0 = sim.sample_populations(nodes)
    n = p.nx
    # after one step slot i of node x + e_i holds f*_i(x)
    tf = np.array([[_neighbor(n, x, ef[i]) for i in range(qf)] for x in nodes])
    tg = np.array([[_neighbor(n, x, eg[i]) for i in range(qg)] for x in nodes])
    sim.step(1)
    allnodes = np.unique(np.concatenate([tf.ravel(), tg.ravel()]))
    fs, gs = sim.sample_populations(allnodes)
    pos = {v: k for k, v in enumerate(allnodes)}
    pf, pg = slot_map(qf), slot_map(qg)
    op = O.lattice_params(1, 1, 1, qf, qg, p.forcing, p.tau_f, p.tau_g, p.G, p.beta, rho0=p.rho0,
                          scalar_mode=p.scalar_mode, sc_shift=p.sc_shift)
    one = O.OracleSim(op)
    worst = 0.0
    for k, x in enumerate(nodes):
        # oracle order <- library order
        fo = np.empty(qf)
        go = np.empty(qg)
        fo[pf] = f0[k]
        go[pg] = g0[k]
        one.set_populations(fo, go)
        one.step(1)
        fa, ga = one.populations()
        f_star = fa[pf, 0]
        g_star = ga[pg, 0]
        f_gpu = np.array([fs[pos[tf[k, i]], i] for i in range(qf)])
        g_gpu = np.array([gs[pos[tg[k, i]], i] for i in range(qg)])
        df = f_star - wf
        dg = g_star - p.rho0 * wg
        sf, sg = np.max(np.abs(df)), np.max(np.abs(dg))
        tol_f = rel_store * np.abs(df) + 2e-6 * sf + abs_store
        tol_g = rel_store * np.abs(dg) + 2e-6 * sg + abs_store
        ef_ = np.abs(f_gpu - f_star)
        eg_ = np.abs(g_gpu - g_star)
        assert np.all(ef_ <= tol_f), (x, np.max(ef_ / sf))
        assert np.all(eg_ <= tol_g), (x, np.max(eg_ / sg))
        worst = max(worst, float(np.max(ef_ / sf)), float(np.max(eg_ / sg)))
    return worst


STORE_REL = {"fp32": 0.0, "fp16": 2.0 ** -10, "bf16": 2.0 ** -7}
# FP16 deviations below 2^-14 are subnormal: their rounding is absolute, 2^-25 at most
STORE_ABS = {"fp32": 0.0, "fp16": 2.0 ** -24, "bf16": 0.0}


@pytest.mark.parametrize("n,pair,forcing,Re,Fr,storage", [
    (256, "27x19", "sc", 800.0, 0.1, "fp32"),    # the bench workload
    (256, "27x19", "sc", 800.0, 0.1, "fp16"),
    (256, "27x19", "sc", 800.0, 0.1, "bf16"),
    (128, "19x7", "guo", 400.0, 0.5, "fp32"),    # 128^3 stencil/forcing sweep
    (128, "19x7", "sc", 400.0, 0.1, "fp32"),
    (128, "27x19", "guo", 400.0, 0.5, "fp32"),
    (128, "27x19", "sc", 400.0, 0.1, "fp32"),
    (128, "27x19", "edm", 400.0, 0.1, "fp32"),
    (512, "27x19", "sc", 1600.0, 0.1, "fp16"),   # 512^3 capacity case
    (512, "27x19", "sc", 1600.0, 0.1, "fp32"),   # 24.7 GB of populations
])
def test_sampled_parity_full_size(n, pair, forcing, Re, Fr, storage):
    p = lbm.lbm_params_from_physics(n, n, n, pair, forcing, Re, Fr, 1.0, 0.04)
    sim = lbm.Simulation(p, storage=storage)
    sim.init_tgv(seed=1, noise_amp=1e-3)
    sim.step(100)  # develop non-equilibrium parts; layout parity even
    nodes = _sample_nodes(n, 160, seed=n)
    w_even = _check_one_step(sim, p, nodes, STORE_REL[storage], STORE_ABS[storage])   # even -> odd
    w_odd = _check_one_step(sim, p, nodes, STORE_REL[storage], STORE_ABS[storage])    # odd -> even
    assert max(w_even, w_odd) < {"fp32": 1e-5, "fp16": 1e-3, "bf16": 8e-3}[storage]
    sim.close()


@pytest.mark.parametrize("n,storage", [(256, "fp32"), (512, "fp16")])
def test_invariants_full_size(n, storage):
    """Mass conserved; lattice momentum gains sum_x F = -G sum rho' per step."""
    p = lbm.lbm_params_from_physics(n, n, n, "27x19", "sc", 800.0 * n / 256, 0.1, 1.0, 0.04)
    sim = lbm.Simulation(p, storage=storage)
    sim.init_tgv(seed=1, noise_amp=1e-3)
    sim.step(50)
    d0 = sim.diagnostics()
    _, _, rp = sim.fields()
    Fz = -p.G * rp.sum()
    sim.step(1)
    d1 = sim.diagnostics()
    n3 = n ** 3
    assert abs(d1["mass_f"] - d0["mass_f"]) / n3 < (1e-9 if storage == "fp32" else 1e-5)
    assert abs((d1["mom_z"] - d0["mom_z"]) - Fz) < (1e-9 if storage == "fp32" else 1e-5) * n3
    assert abs(d1["mom_x"] - d0["mom_x"]) < (1e-9 if storage == "fp32" else 1e-5) * n3
    sim.close()
