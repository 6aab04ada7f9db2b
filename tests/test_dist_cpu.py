"""The bench's multi-process path on CPU (gloo, world size 2): replicas
exchange no lattice data; the job's time is the slowest rank's, the
throughput every rank's updates over it, and under torchrun only rank 0 of
the reference arm does work and prints."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    w, r, _ = bench.dist_setup()
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    # rank r took 1.5 + r seconds: the job time is the slowest rank's
    t = bench.max_over_ranks(w, 1.5 + r)
    value = bench.aggregate_mlups(4.0e6, w, t)
    # the reference arm: ranks other than 0 return without work or output
    out = io.StringIO()
    if r != 0:
        class A:
            steps, warmup = 1, 0
        with redirect_stdout(out):
            bench.run_reference_arm(A)
    bench.barrier(w)
    dist.destroy_process_group()
    q.put((r, t, value, out.getvalue()))


def test_two_gloo_ranks_max_time_and_aggregate():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, t, value, out in res:
        assert t == pytest.approx(2.5)
        assert value == pytest.approx(4.0e6 * 2 / 2.5 / 1e6)
    assert res[1][3] == ""


# ---- the batch sweep split over ranks (no data-path communication) ---------

SWEEP_CPU = [  # small stand-ins of the sweep's instances: (n, pair, forcing, Re, Fr)
    (8, "27x19", "guo", 200.0, 1.0), (6, "19x7", "sc", 200.0, 0.5), (4, "27x19", "sc", 200.0, 0.2),
    (7, "19x7", "guo", 200.0, 0.1), (5, "27x19", "guo", 200.0, 0.5), (6, "27x19", "sc", 200.0, 1.0),
    (4, "19x7", "sc", 200.0, 0.2),
]


def _sweep_params():
    sys.path.insert(0, ROOT)
    from paper_2605_14505_gb300 import lbm

    return [lbm.lbm_params_from_physics(n, n, n, pair, f, Re, Fr, 1.0, 0.04) for n, pair, f, Re, Fr in SWEEP_CPU]


def _oracle_instance(p, steps=3):
    """CPU stand-in for one instance's update: the FP64 oracle (tests only)."""
    sys.path.insert(0, ROOT)
    import stgv_inputs as I
    from oracle import oracle as O
    from paper_2605_14505_gb300 import lbm

    qf, qg = lbm.PAIR_Q[p.pair]
    o = O.OracleSim(O.lattice_params(p.nx, p.ny, p.nz, qf, qg, p.forcing, p.tau_f, p.tau_g, p.G, p.beta,
                                     rho0=p.rho0))
    o.init_fields(*I.tgv_fields(p.nx, 0.04, seed=3, noise_amp=0.01))
    o.step(steps)
    d = o.diagnostics()
    o.close()
    return d


def test_partition_covers_every_instance_once_and_balances_bytes():
    sys.path.insert(0, ROOT)
    from paper_2605_14505_gb300 import lbm

    params = _sweep_params()
    for nranks in (1, 2, 3, 8):
        owner, imb = lbm.lbm_batch_partition(params, nranks)
        assert len(owner) == len(params) and all(0 <= r < nranks for r in owner)
        bytes_ = [(sum(lbm.PAIR_Q[p.pair])) * p.nx * p.ny * p.nz * 4 for p in params]
        load = [sum(b for b, r in zip(bytes_, owner) if r == k) for k in range(nranks)]
        assert imb == pytest.approx(max(load) / (sum(load) / nranks))
        # longest-first greedy: no rank carries more than the mean plus the largest instance
        assert max(load) <= sum(load) / nranks + max(bytes_)
        # deterministic: the same table on every call (every rank computes it alone)
        assert lbm.lbm_batch_partition(params, nranks)[0] == owner
    # one rank owns everything
    assert set(lbm.lbm_batch_partition(params, 1)[0]) == {0}
    with pytest.raises(lbm.LbmError):
        lbm.lbm_batch_partition(params, 0)


def _sweep_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_2605_14505_gb300 import lbm

    w, r, _ = bench.dist_setup()
    params = _sweep_params()
    owner, _ = lbm.lbm_batch_partition(params, w)
    mine = {i: _oracle_instance(params[i]) for i in range(len(params)) if owner[i] == r}
    # reporting only: the per-instance records are gathered once at the end
    gathered = [None] * w
    dist.all_gather_object(gathered, mine)
    dist.destroy_process_group()
    q.put((r, sorted(mine), gathered))


def test_two_gloo_ranks_split_the_sweep_without_exchanging_lattice_data():
    """Each rank updates only the instances lbm_batch_partition gives it; the
    records gathered at the end equal a one-process run of every instance,
    bit for bit, and every instance was updated by exactly one rank."""
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sweep_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    owned = res[0][1] + res[1][1]
    assert sorted(owned) == list(range(len(SWEEP_CPU)))
    assert res[0][1] and res[1][1]
    merged = {}
    for part in res[0][2]:
        merged.update(part)
    params = _sweep_params()
    for i, p in enumerate(params):
        solo = _oracle_instance(p)
        assert merged[i] == solo, i
