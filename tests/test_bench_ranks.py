"""The N > 1 path of bench.py (independent replicas, one per GPU) on CPU:
two gloo ranks report different step times; both get the slowest one, and
the whole-job throughput counts the solves of both ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        ms = [20.0, 25.0][rank]
        got = bench.aggregate_over_ranks(ms, w)
        q.put((r, w, lr, got))
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, w, local, (ms, value)) in enumerate(res):
        assert (rank, w, local) == (r, world, r)
        assert ms == 25.0                       # the slowest rank's step
        assert value == pytest.approx(2 * 1000.0 / 25.0)


def test_aggregate_single_rank():
    import bench
    assert bench.aggregate_over_ranks(10.0, 1) == (10.0, 100.0)
