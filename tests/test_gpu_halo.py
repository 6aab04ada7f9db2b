"""z-slab decomposition on the GPU through the C ABI: a lattice split along z
into two slabs (lbm_set_slab, ghost planes), stepped one step at a time with
the halo exchange of lbm_halo_pack / lbm_halo_unpack around every odd step
(paper_2605_14505_gb300.halo.LocalSlabs: both slabs in this process, buffers
copied on the device; no kernel waits for another), equals the whole periodic
lattice bit for bit: the per-node arithmetic is the same kernel's, and the
exchange moves exactly the slots the odd step reads and writes across the cut.
Multi-GPU runs of the same schedule (SlabExchange over NCCL) are not measured
here: every run has one GPU."""
import numpy as np
import pytest

import stgv_inputs as I
from paper_2605_14505_gb300 import halo, lbm

from _helpers import lattice_params

pytestmark = pytest.mark.gpu

LAM = 2.0 ** -10


def _whole_and_slabs(storage, pair, nx=16, ny=12, nz=12, cuts=(0, 5, 12)):
    N = 3e-3
    p = lattice_params(nx, ny, nz, pair, "sc", 0.53, 0.56, N * LAM, -N / LAM)
    whole = lbm.Simulation(p, storage=storage)
    n3 = nx * ny * nz
    rho, u, rp = I.random_fields(nx, ny, nz, 9, 0.05, 0.01, 0.02 / LAM)
    whole.init_fields(rho, u, rp, I.neq_noise(n3, 10), I.neq_noise(n3, 11), 1e-3)
    f, g = whole.populations()
    qf, qg = whole.qf, whole.qg
    f = f.reshape(qf, nz, ny, nx)
    g = g.reshape(qg, nz, ny, nx)
    slabs = []
    for z0, z1 in zip(cuts[:-1], cuts[1:]):
        zs = np.arange(z0 - 1, z1 + 1) % nz
        ps = lattice_params(nx, ny, len(zs), pair, "sc", 0.53, 0.56, N * LAM, -N / LAM)
        s = lbm.Simulation(ps, storage=storage)
        s.set_populations(f[:, zs].reshape(qf, -1), g[:, zs].reshape(qg, -1))
        slabs.append(s)
    return whole, slabs


def _own(sim, nx, ny):
    f, g = sim.populations()
    nzl = sim.params.nz
    f = f.reshape(sim.qf, nzl, ny, nx)[:, 1:-1]
    g = g.reshape(sim.qg, nzl, ny, nx)[:, 1:-1]
    return f, g


@pytest.mark.parametrize("storage,pair", [("fp32", "27x19"), ("fp16", "27x19"), ("fp32", "19x7")])
def test_two_slabs_equal_the_whole_lattice(storage, pair):
    nx, ny, nz = 16, 12, 12
    whole, slabs = _whole_and_slabs(storage, pair)
    run = halo.LocalSlabs([halo.LibrarySlab(s) for s in slabs])
    assert lbm.lbm_halo_bytes(slabs[0].h) == (9 + 5 if pair == "27x19" else 5 + 1) * nx * ny * \
        (4 if storage == "fp32" else 2)
    done = 0
    for steps in (2, 5, 4):
        whole.step(steps)
        run.step(steps)
        done += steps
        if done % 2:
            run.refresh_ghosts()
        fw, gw = whole.populations()
        fw = fw.reshape(whole.qf, nz, ny, nx)
        gw = gw.reshape(whole.qg, nz, ny, nx)
        fs = np.concatenate([_own(s, nx, ny)[0] for s in slabs], axis=1)
        gs = np.concatenate([_own(s, nx, ny)[1] for s in slabs], axis=1)
        assert np.array_equal(fs, fw) and np.array_equal(gs, gw), (storage, pair, done)
    # diagnostics over the own planes, combined by node count, equal the whole lattice's
    run.refresh_ghosts()
    dw = whole.diagnostics()
    ds = [s.diagnostics() for s in slabs]
    nodes = [(s.params.nz - 2) * nx * ny for s in slabs]
    for key in ("Ek", "Ep", "eps_k"):
        comb = sum(d[key] * n for d, n in zip(ds, nodes)) / sum(nodes)
        assert comb == pytest.approx(dw[key], rel=1e-9), key
    assert np.isnan(ds[0]["eps_p"]) and np.isnan(ds[0]["eps_k_curl"])
    for s in slabs + [whole]:
        s.close()


def test_slab_mode_rejects_what_it_cannot_do():
    p = lattice_params(8, 8, 2, "27x19", "guo", 0.6, 0.6, 1e-5, -4.0)
    s = lbm.Simulation(p)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_set_slab(s.h, True)            # needs nz >= 3
    assert ei.value.code == -1
    p = lattice_params(8, 8, 8, "27x19", "guo", 0.6, 0.6, 1e-5, -4.0)
    s = lbm.Simulation(p)
    buf = np.zeros(1)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_halo_pack(s.h, 0, buf.ctypes.data, buf.ctypes.data)   # not in slab mode
    assert ei.value.code == -7
    lbm.lbm_set_slab(s.h, True)
    with pytest.raises(lbm.LbmError):
        s.init_tgv(1, 0.0)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_halo_pack(s.h, 2, buf.ctypes.data, buf.ctypes.data)
    assert ei.value.code == -1
    # host memory is refused before any copy
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_halo_pack(s.h, 0, buf.ctypes.data, buf.ctypes.data)
    assert ei.value.code == -1
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_halo_unpack(s.h, 1, buf.ctypes.data, buf.ctypes.data)
    assert ei.value.code == -1
