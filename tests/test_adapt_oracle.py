"""Pins for the ADAPT-VQE oracle (Sec. II.C, Fig. 1; BFGS-2 / BFGS-2F of
Sec. IV.D), each independent of the oracle's own code:

* the first iteration against the reference's 2x2 eigenproblem with the
  excitation of largest |<HF|H|D>| (dense Jordan-Wigner Hamiltonian);
* BFGS-2's first step against the minimum of the exact one-parameter energy
  E(t) = A + B cos t + C sin t + D cos 2t + F sin 2t, fitted from dense
  statevector energies;
* the variational bound against dense FCI, monotone energies, the final
  state against the dense statevector of the chosen circuit;
* BFGS-2F leaves earlier parameters untouched; stopping rules.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import jw_dense as J
import oracle as O
from oracle.adapt import OracleAdapt, bootstrap
from paper_2411_07920_gb300 import inputs as I


@pytest.fixture(scope="module")
def c1():
    w = I.workload("so12_e4")
    basis = J.sector(w.n_so, w.n_e)
    H = J.hamiltonian_sector(w.n_so, w.h, w.g, basis)
    return w, basis, H


def _dense_energy(w, basis, H, ops, theta):
    a = J.annihilators(w.n_so)
    psi = np.zeros(1 << w.n_so)
    psi[(1 << w.n_e) - 1] = 1.0
    for op, th in zip(ops, theta):
        psi = spla.expm_multiply(th * J.kappa_matrix(a, op), psi)
    v = psi[basis]
    return float(v @ H @ v / (v @ v))


def test_first_iteration_is_the_two_level_ground_state(c1):
    w, basis, H = c1
    hf = (1 << w.n_e) - 1
    idx = {int(b): i for i, b in enumerate(basis)}
    aops = J.annihilators(w.n_so)
    e0 = np.zeros(1 << w.n_so)
    e0[hf] = 1.0
    pool = O.pool_ops(w.n_so)
    grad, partner = np.zeros(len(pool)), {}
    for k, op in enumerate(pool):
        t = J.tau_matrix(aops, op)
        for vec, sgn in ((t @ e0, 1.0), (t.T @ e0, -1.0)):
            if vec.any():
                d = int(np.flatnonzero(vec)[0])
                grad[k] = 2 * sgn * vec[d] * H[idx[hf], idx[d]]
                partner[k] = d
                break
    top = np.abs(grad).max()
    k_ref = int(np.flatnonzero(np.abs(grad) >= top * (1 - 1e-5))[0])
    d = partner[k_ref]
    block = np.array([[H[idx[hf], idx[hf]], H[idx[hf], idx[d]]], [H[idx[d], idx[hf]], H[idx[d], idx[d]]]])
    a = OracleAdapt(w.n_so, w.n_e, w.h, w.g, 0, eps=1e-3, gtol=1e-10)
    assert a.iterate("bfgs")
    assert a.chosen == [k_ref]
    assert abs(a.energies[0] - np.linalg.eigvalsh(block)[0]) < 1e-10
    assert abs(a.grad_norms[0] - np.linalg.norm(grad)) < 1e-12


def test_bfgs2_first_step_is_the_exact_one_parameter_minimum(c1):
    w, basis, H = c1
    a = OracleAdapt(w.n_so, w.n_e, w.h, w.g, 0, eps=1e-3, gtol=1e-10)
    a.run(3, "bfgs")
    g = a.pool_gradient()
    k = int(np.argmax(np.abs(g)))
    ops = np.concatenate([a.ops, a.pool[k][None, :]])
    theta = a._bfgs_last(np.append(a.theta, 0.0), a.chosen + [k])
    t_star = theta[-1]

    def e_of(t):
        return _dense_energy(w, basis, H, ops, np.append(a.theta, t))
    ts = np.array([0.0, 1.0, -1.0, 2.0, -2.0])
    M = np.stack([np.ones(5), np.cos(ts), np.sin(ts), np.cos(2 * ts), np.sin(2 * ts)], axis=1)
    coef = np.linalg.solve(M, [e_of(t) for t in ts])

    def fit(t):
        return coef @ np.array([1, math.cos(t), math.sin(t), math.cos(2 * t), math.sin(2 * t)])

    def dfit(t):
        return coef @ np.array([0, -math.sin(t), math.cos(t), -2 * math.sin(2 * t), 2 * math.cos(2 * t)])

    def d2fit(t):
        return coef @ np.array([0, -math.cos(t), -math.sin(t), -4 * math.cos(2 * t), -4 * math.sin(2 * t)])
    assert abs(fit(0.3) - e_of(0.3)) < 1e-12  # the five-term form is exact
    t = t_star
    for _ in range(50):  # Newton on the exact fit from the optimiser's answer
        t -= dfit(t) / d2fit(t)
    assert d2fit(t) > 0 and abs(t - t_star) < 1e-7
    assert fit(t) < fit(0.0) - 1e-6
    assert abs(e_of(t_star) - fit(t)) < 1e-12
    assert np.array_equal(theta[:-1], a.theta)  # the others stayed frozen


def test_energies_variational_monotone_and_match_the_statevector(c1):
    w, basis, H = c1
    efci = np.linalg.eigvalsh(H)[0]
    a = OracleAdapt(w.n_so, w.n_e, w.h, w.g, 0, eps=1e-3)
    a.run(10, "bfgs")
    e = np.array(a.energies)
    assert len(e) == 10
    assert np.all(np.diff(e) < 0)
    assert e.min() >= efci - 1e-12
    assert abs(e[-1] - _dense_energy(w, basis, H, a.ops, a.theta)) < 1e-12
    # each VQE converged: the oracle's gradient at the optimum is below gtol (plus rounding)
    _, d = O.energy_grad(w.n_so, w.n_e, w.h, w.g, a.ops, a.theta, 0)
    assert np.abs(d).max() < 1e-5


def test_bfgs2f_keeps_earlier_parameters_frozen(c1):
    w, basis, H = c1
    a = OracleAdapt(w.n_so, w.n_e, w.h, w.g, 0, eps=1e-3)
    a.run(3, "bfgs2")
    for _ in range(3):
        before = a.theta.copy()
        e_prev = a.energies[-1]
        assert a.iterate("bfgs2f")
        assert np.array_equal(a.theta[:len(before)], before)
        assert a.energies[-1] < e_prev


def test_stopping_rules_and_bootstrap(c1):
    w, basis, H = c1
    # converged at once: ||g|| below a large eps
    a = OracleAdapt(w.n_so, w.n_e, w.h, w.g, 0, eps=10.0)
    assert a.run(5, "bfgs") and len(a.theta) == 0 and a.grad_norms[0] < 10.0
    # a small N_CUT fills up; then the chosen operator's fixed-projector
    # derivative at 0 is exactly zero, nothing improves, the run stalls
    a = OracleAdapt(w.n_so, w.n_e, w.h, w.g, 6, eps=1e-4)
    assert not a.run(40, "bfgs") and a.stalled
    n = len(a.theta)
    keys, _ = O.apply_ansatz(w.n_so, w.n_e, a.ops, a.theta, 6)
    assert len(keys) == 6
    k = O.pool_gradients(w.n_so, w.h, w.g, *O.apply_ansatz(w.n_so, w.n_e, a.ops, a.theta, 6))
    k = int(np.flatnonzero(np.abs(k) >= np.abs(k).max() * (1 - 1e-5))[0])
    _, d = O.energy_grad(w.n_so, w.n_e, w.h, w.g, np.concatenate([a.ops, a.pool[k][None, :]]),
                         np.append(a.theta, 0.0), 6)
    assert d[-1] == 0.0
    # a bootstrap continues the same ansatz at larger N_CUT and lowers E further
    b, stages = bootstrap(w.n_so, w.n_e, w.h, w.g, [6, 20, 60], 40, eps=1e-4)
    assert [s["n_keep"] for s in stages] == [6, 20, 60]
    assert stages[0]["n_params"] == n
    assert stages[1]["n_params"] > stages[0]["n_params"] and stages[2]["n_params"] >= stages[1]["n_params"]
    assert b.energies[-1] < a.energies[-1]
