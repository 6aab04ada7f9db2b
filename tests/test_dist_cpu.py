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
