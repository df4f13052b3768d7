"""The benchmark's multi-rank path (replicas, max-over-ranks timing) on CPU
with the gloo backend, world size 2."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total_ms = [800.0, 1200.0][rank]  # rank 1 is the slow one
    ms, value = bench.aggregate(total_ms, 4, world, torch.device("cpu"))
    q.put((rank, ms, value, bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_takes_the_slowest_rank_and_counts_all_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, env in out:
        assert ms == pytest.approx(1200.0 / 4)
        assert value == pytest.approx(2 * 4 / 1.2)  # both ranks' sweeps over the slowest rank's time
        assert env[0] == rank and env[1] == 2
