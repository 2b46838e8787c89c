"""The multi-GPU path is replicas only (one independent halo per rank, no
data-path collective): the benchmark's cross-rank aggregation takes the
slowest rank's time and sums the work.  Checked with world size 2 on gloo
(CPU)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, counts = bench.combine_ranks(100.0 + 50.0 * rank, (1000 + rank, 10 * (rank + 1)))
    out.put((rank, ms, counts))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, counts in res:
        assert ms == 150.0                    # slowest rank
        assert counts == [2001.0, 30.0]       # summed work


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(12.5, (3, 4)) == (12.5, [3, 4])
