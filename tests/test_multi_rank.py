"""The N > 1 path of bench.py (independent replicas, one per GPU) on CPU:
two gloo ranks aggregate their timed spans and work the way the benchmark
does (slowest rank's time, work of all ranks)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env()[:2] == (rank, world)
    elapsed, work = bench.aggregate_ranks(1.0 + rank, 10.0 * (rank + 1), "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, elapsed, work))


def test_two_replicas_aggregate_with_gloo():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    # both ranks see the slowest span (2 s) and the total work (30)
    assert res == [(0, 2.0, 30.0), (1, 2.0, 30.0)]
