"""MP2-ordered UCCSD guess and the overlap / infidelity through the library
against the oracle (oracle/uccsd.py)."""
import numpy as np
import pytest

import oracle as O
from oracle.uccsd import infidelity, mp2_uccsd, overlap
from paper_2411_07920_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2411_07920_gb300 import swcs
    return swcs


@pytest.mark.parametrize("name", ["so12_e4", "so28_e8", "so52_e12"])
def test_mp2_uccsd_matches_oracle(S, name):
    w = I.workload(name)
    c = S.Context()
    c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    ops, theta = c.mp2_uccsd()
    ops_o, theta_o = mp2_uccsd(w.h, w.g, w.n_so, w.n_e)
    assert np.array_equal(ops, ops_o)
    assert np.abs(theta - theta_o).max() <= 1e-15 * np.abs(theta_o).max()
    if w.n_so <= 28:  # the guess as an ansatz: same state and energy as the oracle's
        n_keep = 0 if w.n_so == 12 else 20000
        c.apply_ansatz(ops, theta, n_keep)
        k, a = c.get_state()
        ko, ao = O.apply_ansatz(w.n_so, w.n_e, ops_o, theta_o, n_keep)
        assert np.array_equal(k, ko) and np.abs(a - ao).max() < 1e-14
        assert abs(c.energy()[0] - O.energy(w.n_so, w.h, w.g, ko, ao)[0]) < 1e-10


@pytest.mark.parametrize("n_so,n_e,n_keep", [(12, 4, 0), (20, 6, 300), (28, 8, 3000)])
def test_overlap_and_infidelity_match_oracle(S, n_so, n_e, n_keep):
    w = I.small_case(n_so, n_e, 30, 170 + n_so, n_keep=n_keep)
    c = S.Context()
    c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    c.apply_ansatz(w.ops, w.theta, n_keep)
    ka, aa = O.apply_ansatz(n_so, n_e, w.ops, w.theta, n_keep)
    kb, ab = O.apply_ansatz(n_so, n_e, w.ops[: len(w.ops) // 2], w.theta[: len(w.ops) // 2] * 1.3, n_keep)
    ov, na, nb, inf = c.overlap(kb, ab)
    assert abs(ov - overlap(ka, aa, kb, ab)) < 1e-13
    assert abs(na - float(aa @ aa)) < 1e-13 and abs(nb - float(ab @ ab)) < 1e-13
    assert abs(inf - infidelity(ka, aa, kb, ab)) < 1e-12
    assert abs(c.overlap(ka, aa)[3]) < 1e-13                      # with itself
    assert c.overlap(np.zeros(0, np.uint64), np.zeros(0))[0] == 0.0  # empty given state


def test_uccsd_vqe_matches_oracle(S):
    from oracle.uccsd import vqe as oracle_vqe
    from paper_2411_07920_gb300 import adapt
    w = I.workload("so12_e4")
    c = S.Context()
    c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    ops, theta = c.mp2_uccsd()
    e, th, calls = adapt.vqe(c, ops, theta, 0)
    eo, tho = oracle_vqe(w.n_so, w.n_e, w.h, w.g, ops, theta, 0)
    assert calls > 1
    assert abs(e - eo) < 1e-9
