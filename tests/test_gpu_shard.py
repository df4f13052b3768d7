"""The pool sweep in shards (swcs_pool_gradients_partial_dev) on one GPU: every
shard against the oracle's shard (pairs whose E has its alpha string's colex
rank = shard mod n), and the shards' sum against the whole sweep and the
oracle; the host helper through a one-rank NCCL group."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2411_07920_gb300 import inputs as I

import pool_ref as R

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.mark.parametrize("n_so,n_e,n_ops,seed,n_keep,check_each", [
    (12, 4, 10, 1, 0, True), (16, 6, 30, 71, 60, True), (28, 8, 60, 2, 3000, False)])
@pytest.mark.parametrize("n_shards", [2, 3])
def test_shards_partition_the_sweep(n_so, n_e, n_ops, seed, n_keep, check_each, n_shards):
    import torch
    from paper_2411_07920_gb300 import swcs
    w = I.small_case(n_so, n_e, n_ops, seed, n_keep=n_keep)
    with swcs.Context() as c:
        c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
        c.apply_ansatz(w.ops, w.theta, n_keep)
        k, a = c.get_state()
        P = c.pool_size()
        pool = c.pool_ops()
        tot = np.zeros(P)
        num = 0.0
        for s in range(n_shards):
            graw = torch.empty(P, dtype=torch.float64, device="cuda")
            acc = torch.empty(2, dtype=torch.float64, device="cuda")
            c.pool_gradients_partial_dev(s, n_shards, graw, acc)
            torch.cuda.synchronize()
            g_s, (num_s, n2) = graw.cpu().numpy(), acc.tolist()
            assert abs(n2 - a @ a) < 1e-13
            if check_each:
                go_s, numo_s, _ = R.shard_partial(w.n_so, pool, k, a,
                                                  lambda at: O.sigma_at(w.n_so, w.h, w.g, k, a, at), s, n_shards)
                assert np.abs(g_s - go_s).max() < TOL
                assert abs(num_s - numo_s) < TOL
            tot += g_s
            num += num_s
        g = c.pool_gradients()
        e, _ = c.sweep_energy()
        assert np.abs(2.0 * tot / (a @ a) - g).max() < TOL
        assert abs(num / (a @ a) - e) < TOL
        go = O.pool_gradients(w.n_so, w.h, w.g, k, a)
        assert np.abs(g - go).max() < TOL


def test_partial_rejects_bad_shards():
    import torch
    from paper_2411_07920_gb300 import swcs
    w = I.small_case(12, 4, 10, 1)
    with swcs.Context() as c:
        c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
        c.apply_ansatz(w.ops, w.theta, 0)
        t = torch.empty(c.pool_size() + 2, dtype=torch.float64, device="cuda")
        for s, n in ((2, 2), (-1, 2), (0, 0)):
            with pytest.raises(swcs.SwcsError):
                c.pool_gradients_partial_dev(s, n, t, t)


def test_host_helper_on_a_one_rank_group():
    import torch
    import torch.distributed as dist
    from paper_2411_07920_gb300 import shard, swcs
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        w = I.small_case(28, 8, 60, 2, n_keep=3000)
        with swcs.Context() as c:
            c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
            c.apply_ansatz(w.ops, w.theta, 3000)
            g, e = shard.sharded_pool_gradients(c)
            g0 = c.pool_gradients()
            e0, _ = c.sweep_energy()
        assert np.abs(g.cpu().numpy() - g0).max() < TOL
        assert abs(e - e0) < TOL
    finally:
        dist.destroy_process_group()
