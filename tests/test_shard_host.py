"""The sharded pool sweep's host side on CPU: two gloo ranks, each with a
stand-in context whose shard is computed by the oracle (sigma pulled per
determinant), summed by paper_2411_07920_gb300.shard's all-reduce.  The
shards must partition the sweep exactly: the sum equals the oracle's full
pool gradient and energy."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as O
from paper_2411_07920_gb300 import inputs as I

import pool_ref as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASE = (16, 6, 30, 71, 60)  # n_so, n_e, gates, seed, N


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class OracleShardContext:
    """Stand-in for swcs.Context: pool_size and pool_gradients_partial_dev from the oracle."""

    def __init__(self, w, keys, amps):
        self.w, self.keys, self.amps = w, keys, amps
        self.pool = O.pool_ops(w.n_so)

    def pool_size(self):
        return len(self.pool)

    def pool_gradients_partial_dev(self, shard, n_shards, d_graw, d_acc):
        import torch
        w = self.w
        graw, num, n2 = R.shard_partial(w.n_so, self.pool, self.keys, self.amps,
                                        lambda at: O.sigma_at(w.n_so, w.h, w.g, self.keys, self.amps, at),
                                        shard, n_shards)
        d_graw.copy_(torch.from_numpy(graw))
        d_acc[0] = num
        d_acc[1] = n2


def _worker(rank, world, port, q):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2411_07920_gb300 import shard
    n_so, n_e, n_ops, seed, n_keep = CASE
    w = I.small_case(n_so, n_e, n_ops, seed, n_keep=n_keep)
    k, a = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_keep)
    g, e = shard.sharded_pool_gradients(OracleShardContext(w, k, a))
    q.put((rank, g.numpy(), e))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_sum_to_the_full_sweep_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n_so, n_e, n_ops, seed, n_keep = CASE
    w = I.small_case(n_so, n_e, n_ops, seed, n_keep=n_keep)
    k, a = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_keep)
    go = O.pool_gradients(w.n_so, w.h, w.g, k, a)
    eo, _ = O.energy(w.n_so, w.h, w.g, k, a)
    for rank, g, e in out:
        assert np.abs(g - go).max() < 1e-12
        assert abs(e - eo) < 1e-12


def test_each_shard_is_a_proper_part():
    """Every shard holds a nonzero share, and the owners of a pair's E are one rank."""
    n_so, n_e, n_ops, seed, n_keep = CASE
    w = I.small_case(n_so, n_e, n_ops, seed, n_keep=n_keep)
    k, a = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_keep)
    pool = O.pool_ops(w.n_so)
    sig = lambda at: O.sigma_at(w.n_so, w.h, w.g, k, a, at)  # noqa: E731
    parts = [R.shard_partial(w.n_so, pool, k, a, sig, s, 3) for s in range(3)]
    for graw, num, _ in parts:
        assert np.abs(graw).max() > 1e-6
    tot = sum(p[0] for p in parts)
    assert np.abs(2.0 * tot / (a @ a) - O.pool_gradients(w.n_so, w.h, w.g, k, a)).max() < 1e-12
    assert abs(sum(p[1] for p in parts) / (a @ a) - O.energy(w.n_so, w.h, w.g, k, a)[0]) < 1e-12
