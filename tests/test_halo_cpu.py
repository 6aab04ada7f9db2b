"""The z-slab halo exchange schedule (paper_2605_14505_gb300.halo) on CPU, with
the node-local AA stand-in of tests/_slab_cpu.py in place of the library's
kernels: a lattice split along z into slabs that exchange their e_z != 0
slots around every odd step equals the whole periodic lattice, bit for bit,
in one process (LocalSlabs) and over two gloo ranks (SlabExchange)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from _slab_cpu import NumpyAA, slabs_of  # noqa: E402
from paper_2605_14505_gb300 import halo  # noqa: E402


def _initial(q=19, nz=10, ny=6, nx=7, seed=5):
    rng = np.random.default_rng(seed)
    return 0.05 + 0.01 * rng.standard_normal((q, nz, ny, nx))


def _whole(f, steps, q=19):
    w = NumpyAA(f, q)
    for _ in range(steps):
        w.step()
    return w


@pytest.mark.parametrize("q", [19, 27, 7])
@pytest.mark.parametrize("nranks", [1, 2, 3])
def test_local_slabs_equal_the_whole_lattice(q, nranks):
    f = _initial(q)
    for steps in (2, 5, 8):
        ref = _whole(f, steps, q)
        parts = slabs_of(f, nranks)
        backs = [NumpyAA(p[2], q, slab=True) for p in parts]
        run = halo.LocalSlabs(backs)
        run.step(steps)
        if steps % 2:
            # the layout keeps populations at neighbour locations: the ghost
            # planes must hold the neighbours' current slots before a read;
            # the own planes' cells themselves already match
            run.refresh_ghosts()
        got = np.concatenate([b.f[:, 1:-1] for b in backs], axis=1)
        assert np.array_equal(got, ref.f), (q, nranks, steps)


def test_a_slab_without_exchange_differs():
    """The exchange matters: stepping the slabs without it breaks the result
    at the boundary planes (odd steps only)."""
    f = _initial()
    ref = _whole(f, 2)
    parts = slabs_of(f, 2)
    backs = [NumpyAA(p[2], 19, slab=True) for p in parts]
    for b in backs:
        b.step()
        b.step()
    got = np.concatenate([b.f[:, 1:-1] for b in backs], axis=1)
    assert not np.array_equal(got, ref.f)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, steps, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist

    from _slab_cpu import NumpyAA, slabs_of
    from paper_2605_14505_gb300 import halo

    dist.init_process_group("gloo")
    parts = slabs_of(_initial(q), world)
    b = NumpyAA(parts[rank][2], q, slab=True)
    ex = halo.SlabExchange(b, rank, world)
    ex.step(steps)
    own = b.f[:, 1:-1]
    got = [None] * world
    dist.all_gather_object(got, own)
    dist.destroy_process_group()
    if rank == 0:
        np.save(os.environ["SLAB_OUT"], np.concatenate(got, axis=1))


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_halos(tmp_path, world):
    import torch.multiprocessing as mp

    q, steps = 27, 6
    out = str(tmp_path / "slabs.npy")
    os.environ["SLAB_OUT"] = out
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert np.array_equal(np.load(out), _whole(_initial(q), steps, q).f)
