"""The multi-rank path of bench.py (replicas, max-over-ranks timing) on CPU with gloo."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    mx = bench.allreduce_max(ms, world)
    v = bench.aggregate(world, 256 ** 3, 10, mx)
    out.put((rank, mx, v))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, v in res:
        assert mx == 150.0
        assert abs(v - 2 * 256 ** 3 * 10 / 0.15 / 1e6) < 1e-6


def test_single_rank_identity():
    import bench
    assert bench.allreduce_max(3.5, 1) == 3.5
    assert abs(bench.aggregate(1, 1000, 2, 1.0) - 2.0) < 1e-12
