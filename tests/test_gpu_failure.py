"""Failure handling on the GPU without faulting it: a bounded device wait is
made to run out on purpose and must come back as SWCS_ERR_TIMEOUT with the
context still usable; an undersized hash table must be regrown."""
import numpy as np
import pytest

import oracle as O
from paper_2411_07920_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def S():
    from paper_2411_07920_gb300 import swcs
    return swcs


def test_bounded_wait_timeout_reports_and_context_recovers(S):
    w = I.small_case(16, 6, 30, 501, n_keep=200)
    c = S.Context()
    c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    c.set_option("wait_timeout_ms", 50)
    c.set_option("test_skip_arrive", 0)  # CTA 0 never arrives: every other CTA's wait runs out
    with pytest.raises(S.SwcsError) as ei:
        c.apply_ansatz(w.ops, w.theta, 200)
    assert ei.value.code == -4
    c.set_option("test_skip_arrive", -1)
    c.set_option("wait_timeout_ms", 2000)
    c.apply_ansatz(w.ops, w.theta, 200)
    k, a = c.get_state()
    ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 200)
    assert np.array_equal(k, ko) and np.array_equal(a, ao)
    c.close()


def test_hashed_sweep_regrows_an_undersized_table(S):
    w = I.small_case(20, 6, 45, 502, n_keep=800)
    c = S.Context()
    c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    c.apply_ansatz(w.ops, w.theta, 800)
    c.set_option("sweep", 1)
    c.set_option("ext_capacity", 2048)
    g = c.pool_gradients()
    st = c.stats()
    assert st["ext_distinct"] > 2048 and st["ext_capacity"] > 2048
    go = O.pool_gradients(w.n_so, w.h, w.g, *O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 800))
    assert np.abs(g - go).max() < TOL
    c.close()


def test_batch_wait_for_work_is_bounded():
    """One instance of a persistent batched launch is never picked up (test
    hook): the others finish, the idle CTAs' wait for work runs out after the
    bound, the run reports SWCS_ERR_TIMEOUT, and the batch then runs normally."""
    from paper_2411_07920_gb300 import swcs
    specs = [(12, 4, 10, 201, 0), (16, 6, 25, 202, 120), (20, 6, 40, 203, 400)]
    ws = [I.small_case(*sp[:4], n_keep=sp[4]) for sp in specs]
    b = swcs.Batch()
    for w in ws:
        b.add(w.h, w.g, w.n_so, w.n_e, w.ops, w.theta, w.n_keep)
    b.set_option("wait_timeout_ms", 100)
    b.set_option("test_stall_instance", 1)
    b.build(autotune=False)
    b.run()
    with pytest.raises(swcs.SwcsError) as ei:
        b.results(0)
    assert ei.value.code == -4  # SWCS_ERR_TIMEOUT
    b.set_option("test_stall_instance", -1)
    b.build(autotune=False)
    b.run()
    for i, w in enumerate(ws):
        e, n2, g = b.results(i)
        ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, w.n_keep)
        assert abs(e - O.energy(w.n_so, w.h, w.g, ko, ao)[0]) < 1e-10
    b.close()
