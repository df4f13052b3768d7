"""Adjoint dE/dtheta of the truncated ansatz on the GPU against the oracle's
adjoint (fixed-projector derivative) and central finite differences of the
GPU's own energy where every kept set is stable under +-h."""
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


@pytest.mark.parametrize("n_so,n_e,n_ops,seed,n_keep,ckpt", [
    (12, 4, 10, 1, 0, 20), (12, 4, 12, 61, 6, 1), (16, 6, 30, 71, 60, 4), (20, 6, 45, 72, 300, 20),
    (28, 8, 60, 104, 3000, 7), (24, 8, 33, 73, 500, 100)])
def test_adjoint_matches_oracle(S, n_so, n_e, n_ops, seed, n_keep, ckpt):
    w = I.small_case(n_so, n_e, n_ops, seed, n_keep=n_keep)
    c = S.Context()
    c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    e, d = c.energy_grad(w.ops, w.theta, n_keep, ckpt)
    eo, do = O.energy_grad(w.n_so, w.n_e, w.h, w.g, w.ops, w.theta, n_keep)
    assert abs(e - eo) < TOL
    assert np.abs(d - do).max() < TOL, np.abs(d - do).max()
    # the context is left holding psi_M
    k, a = c.get_state()
    ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_keep)
    assert np.array_equal(k, ko) and np.array_equal(a, ao)


def test_adjoint_finite_differences(S):
    w = I.small_case(20, 6, 30, 74, n_keep=400)
    c = S.Context()
    c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    _, d = c.energy_grad(w.ops, w.theta, 400, 5)
    h = 1e-5
    checked = 0
    base = []
    for m in range(1, len(w.ops) + 1):
        c.apply_ansatz(w.ops[:m], w.theta[:m], 400)
        base.append(c.get_state()[0])
    for g in range(0, len(w.ops), 3):
        es, stable = [], True
        for sgn in (1, -1):
            th = w.theta.copy()
            th[g] += sgn * h
            for m in range(1, len(w.ops) + 1):
                c.apply_ansatz(w.ops[:m], th[:m], 400)
                if not np.array_equal(c.get_state()[0], base[m - 1]):
                    stable = False
                    break
            if not stable:
                break
            es.append(c.energy()[0])
        if not stable:
            continue
        fd = (es[0] - es[1]) / (2 * h)
        assert abs(fd - d[g]) < 1e-7
        checked += 1
    assert checked >= 5


def test_autograd_function(S):
    import torch
    from paper_2411_07920_gb300.autograd import energy
    w = I.small_case(16, 6, 20, 75, n_keep=80)
    c = S.Context()
    c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    theta = torch.tensor(w.theta, dtype=torch.float64, requires_grad=True)
    e = energy(theta, c, w.ops, 80, 6)
    (g,) = torch.autograd.grad(3.0 * e, theta)
    eo, do = O.energy_grad(w.n_so, w.n_e, w.h, w.g, w.ops, w.theta, 80)
    assert abs(e.item() - eo) < TOL
    assert np.abs(g.numpy() - 3.0 * do).max() < 3 * TOL


@pytest.mark.parametrize("n_so,n_e,n_ops,seed,n_keep,ckpt,zeros", [
    (12, 4, 10, 1, 0, 20, (3, 9)), (12, 4, 10, 1, 0, 4, tuple(range(10))), (16, 6, 30, 71, 60, 4, (0, 13, 29)),
    (20, 6, 45, 72, 300, 20, (44,)), (24, 8, 33, 73, 0, 7, (32,))])
def test_adjoint_at_zero_angles_matches_oracle(S, n_so, n_e, n_ops, seed, n_keep, ckpt, zeros):
    """theta_g = 0 (how ADAPT starts a new parameter): the kept sets of the
    projectors include the gate's zero-amplitude partners."""
    w = I.small_case(n_so, n_e, n_ops, seed, n_keep=n_keep)
    theta = w.theta.copy()
    theta[list(zeros)] = 0.0
    c = S.Context()
    c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    e, d = c.energy_grad(w.ops, theta, n_keep, ckpt)
    eo, do = O.energy_grad(w.n_so, w.n_e, w.h, w.g, w.ops, theta, n_keep)
    assert abs(e - eo) < TOL
    assert np.abs(d - do).max() < TOL, np.abs(d - do).max()
    if n_keep == 0:
        assert all(abs(do[z]) > 1e-8 for z in zeros)  # zero angles, nonzero derivatives
    k, a = c.get_state()
    ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, theta, n_keep)
    assert np.array_equal(k, ko) and np.array_equal(a, ao)
