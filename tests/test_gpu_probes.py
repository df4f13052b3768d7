"""Hash-probe counters (option count_probes): the gate kernel counts one
partner lookup per determinant a gate acts on, the row sweep one alpha-string
lookup per candidate neighbour of every target; slots visited >= lookups; the
results do not change while counting."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2411_07920_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_probe_counts():
    from paper_2411_07920_gb300 import swcs
    w = I.small_case(20, 6, 30, 91, n_keep=400)
    with swcs.Context() as c:
        c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
        c.apply_ansatz(w.ops, w.theta, 400)
        g0 = c.pool_gradients()
        c.set_option("count_probes", 1)
        c.probe_counts(reset=True)
        c.apply_ansatz(w.ops, w.theta, 400)
        k, a = c.get_state()
        g1 = c.pool_gradients()
        pc = c.probe_counts(reset=True)
        assert np.array_equal(g0, g1) or np.abs(g0 - g1).max() < 1e-12
        ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 400)
        assert np.array_equal(k, ko) and np.array_equal(a, ao)
        # the row sweep looks up every single and double alpha excitation of every target alpha string
        m, ks = w.n_so // 2, w.n_e // 2
        n_cand = ks * (m - ks) + math.comb(ks, 2) * math.comb(m - ks, 2)
        assert pc["row_lookups"] == math.comb(m, ks) * n_cand
        assert pc["row_slots"] >= pc["row_lookups"] and pc["gate_slots"] >= pc["gate_lookups"] > 0
        assert c.probe_counts(reset=True)["row_lookups"] == 0
