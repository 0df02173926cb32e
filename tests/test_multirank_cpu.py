"""Rank logic of the multi-GPU bench, run as two gloo ranks on the CPU: the
whole-job reduction (slowest rank's time, summed converged units) and the
round-robin sharding of independent meshes (every mesh on exactly one rank).
The solve itself has no collective: ranks never exchange data."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    el, c = bench.reduce_over_ranks(1.5 + rank, 10 + 3 * rank)  # CPU tensors
    parts = bench.shard(list(range(48)), rank, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, el, c, parts))


def test_two_ranks_reduce_and_shard():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, el, c, parts in res:
        assert el == 2.5 and c == 23.0  # max of 1.5, 2.5; 10 + 13
    a, b = res[0][3], res[1][3]
    assert not set(a) & set(b) and sorted(a + b) == list(range(48))
    assert abs(len(a) - len(b)) <= 1


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(3.0, 7) == (3.0, 7.0)
    assert bench.shard(range(5), 0, 1) == [0, 1, 2, 3, 4]
