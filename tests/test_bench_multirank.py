"""The multi-rank bookkeeping of bench.py on CPU with gloo (world size 2).

Each rank searches its own replicas; the job's figures are the slowest rank's
time and the sum of all ranks' work.  Ranks get distinct seeds.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, ev, mn = bench.job_totals(1.0 + rank, 1000 * (rank + 1), 10 + rank, dist, "cpu")
    seeds = bench.seeds_for("c3", 4, rank)
    out.put((rank, t, ev, mn, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_job_totals_and_rank_seeds_with_gloo():
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
    for rank, t, ev, mn, seeds in res:
        assert t == 2.0            # slowest rank
        assert ev == 3000.0        # 1000 + 2000
        assert mn == 21.0
    assert set(res[0][4]).isdisjoint(res[1][4])
