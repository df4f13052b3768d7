"""Magnitude-threshold truncation (Sec. II.B's alternative criterion) on the
GPU against the oracle: kept sets and amplitudes bit-exact, energies, pool
gradients and the adjoint within 1e-10."""
import math

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


def _ctx(S, w, eps):
    c = S.Context()
    c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    c.set_truncation_threshold(eps)
    return c


@pytest.mark.parametrize("n_so,n_e,n_ops,seed,n_keep,eps", [
    (12, 4, 30, 201, 0, 1e-3), (16, 6, 40, 202, 0, 1e-4), (20, 6, 50, 203, 400, 1e-4),
    (28, 8, 60, 204, 0, 2e-4), (28, 8, 60, 204, 1500, 2e-4), (16, 4, 25, 205, 0, 0.05)])
def test_threshold_gate_sequence_bit_exact(S, n_so, n_e, n_ops, seed, n_keep, eps):
    w = I.small_case(n_so, n_e, n_ops, seed, n_keep=n_keep)
    c = _ctx(S, w, eps)
    c.apply_ansatz(w.ops, w.theta, n_keep)
    k, a = c.get_state()
    ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_keep, eps=eps)
    assert np.array_equal(k, ko) and np.array_equal(a, ao)
    assert len(ko) == 0 or np.abs(ao).min() >= eps
    # the criterion acted: the count-only state differs
    k0, a0 = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_keep)
    assert not (np.array_equal(k0, ko) and np.array_equal(a0, ao))
    e, n2 = c.energy()
    eo, n2o = O.energy(w.n_so, w.h, w.g, ko, ao)
    assert abs(e - eo) < TOL and abs(n2 - n2o) < 1e-13
    if n_so <= 20:
        g = c.pool_gradients()
        go = O.pool_gradients(w.n_so, w.h, w.g, ko, ao)
        assert np.abs(g - go).max() < TOL
    # eps = 0 restores the count-only rule on the same context
    c.set_truncation_threshold(0.0)
    c.apply_ansatz(w.ops, w.theta, n_keep)
    k, a = c.get_state()
    ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_keep)
    assert np.array_equal(k, ko) and np.array_equal(a, ao)


@pytest.mark.parametrize("n_so,n_e,n_ops,seed,n_keep,eps,ckpt", [
    (12, 4, 12, 206, 0, 5e-3, 4), (20, 6, 40, 207, 0, 1e-4, 20), (24, 8, 33, 208, 300, 1e-4, 7)])
def test_threshold_adjoint_matches_oracle(S, n_so, n_e, n_ops, seed, n_keep, eps, ckpt):
    w = I.small_case(n_so, n_e, n_ops, seed, n_keep=n_keep)
    c = _ctx(S, w, eps)
    e, d = c.energy_grad(w.ops, w.theta, n_keep, ckpt)
    eo, do = O.energy_grad(w.n_so, w.n_e, w.h, w.g, w.ops, w.theta, n_keep, eps=eps)
    assert abs(e - eo) < TOL
    assert np.abs(d - do).max() < TOL


def test_threshold_rejects_bad_values(S):
    w = I.small_case(12, 4, 3, 209)
    c = _ctx(S, w, 0.0)
    for bad in (-1e-3, math.nan, math.inf):
        with pytest.raises(S.SwcsError):
            c.set_truncation_threshold(bad)
    # a threshold above every amplitude but the reference's empties nothing it should not:
    # the reference amplitude cos(theta) products stay above 0.5 for these small angles
    c.set_truncation_threshold(0.5)
    c.apply_ansatz(w.ops, w.theta * 0.1, 0)
    k, a = c.get_state()
    ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta * 0.1, 0, eps=0.5)
    assert np.array_equal(k, ko) and np.array_equal(a, ao) and len(k) == 1


def test_empty_state_is_reported_not_computed(S):
    """A threshold above every amplitude empties the state; energies, sweeps
    and the adjoint then report SWCS_ERR_INVALID_ARG instead of running."""
    w = I.small_case(12, 4, 6, 210)
    c = _ctx(S, w, 2.0)
    c.apply_ansatz(w.ops, w.theta, 0)
    k, a = c.get_state()
    assert len(k) == 0 and len(O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 0, eps=2.0)[0]) == 0
    for call in (c.energy, c.pool_gradients, lambda: c.energy_grad(w.ops, w.theta, 0, 4)):
        with pytest.raises(S.SwcsError) as ei:
            call()
        assert ei.value.code == -1
    # an all-zero state set by the caller is empty too
    c.set_truncation_threshold(0.0)
    c.set_state(np.array([0b1111], np.uint64), np.array([0.0]))
    with pytest.raises(S.SwcsError):
        c.energy()
    # the context stays usable
    c.apply_ansatz(w.ops, w.theta, 0)
    e, _ = c.energy()
    ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 0)
    assert abs(e - O.energy(w.n_so, w.h, w.g, ko, ao)[0]) < TOL
