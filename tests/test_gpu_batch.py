"""Batched graph launch: every instance's energy and pool gradient equal the
single-context path and the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2411_07920_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-10

SMALL = [(12, 4, 10, 201, 0), (16, 6, 25, 202, 120), (20, 6, 40, 203, 400), (14, 4, 20, 204, 50),
         (18, 8, 30, 205, 300), (24, 8, 35, 206, 600), (16, 2, 8, 207, 0)]


@pytest.fixture(scope="module")
def S():
    from paper_2411_07920_gb300 import swcs
    return swcs


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_oracle(S, autotune):
    b = S.Batch()
    ws = [I.small_case(n_so, n_e, n_ops, seed, n_keep=nk) for (n_so, n_e, n_ops, seed, nk) in SMALL]
    for w in ws:
        b.add(w.h, w.g, w.n_so, w.n_e, w.ops, w.theta, w.n_keep)
    b.build(autotune=autotune)
    for rep in range(2):
        b.run()
        for i, w in enumerate(ws):
            e, n2, g = b.results(i)
            ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, w.n_keep)
            eo, n2o = O.energy(w.n_so, w.h, w.g, ko, ao)
            go = O.pool_gradients(w.n_so, w.h, w.g, ko, ao)
            assert abs(e - eo) < TOL and abs(n2 - n2o) < 1e-13
            assert np.abs(g - go).max() < TOL
    t = b.tuning()
    assert t["instances"] == len(ws)
    b.close()


def test_batch_uneven_instances_match_single_contexts(S):
    specs = [s for s in I.batch_specs(64, 100) if s["n_so"] <= 24][:10]
    for s in specs:
        s["n_keep"] = min(s["n_keep"], 3000)
        s["n_gates"] = min(s["n_gates"], 60)
    b = S.Batch()
    ws = []
    for s in specs:
        w = I.batch_instance(s)
        ws.append(w)
        b.add(w.h, w.g, w.n_so, w.n_e, w.ops, w.theta, w.n_keep)
    b.build(autotune=True)
    b.run()
    for i, w in enumerate(ws):
        e, n2, g = b.results(i)
        c = S.Context()
        c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
        c.apply_ansatz(w.ops, w.theta, w.n_keep)
        g1 = c.pool_gradients()
        e1, n21 = c.sweep_energy()
        assert abs(e - e1) < TOL and abs(n2 - n21) < 1e-13
        assert np.abs(g - g1).max() < TOL
        c.close()
    b.close()
