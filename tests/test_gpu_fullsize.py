"""Parity at the benchmark's full size (52 spin-orbitals, 12 electrons,
200 gates, N = 1e6) in the launch configuration bench.py times, on outputs
the oracle can compute one at a time:
  * the last gate with its truncation, bit-exact, from the GPU's state after
    199 gates (the oracle's own full run takes minutes);
  * sigma_D on sampled determinants (oracle pulls each from its connections);
  * pool gradients of sampled operators with small support (oracle pull form);
  * properties at any size: N kept determinants, particle number, S_z, the
    energies of the two sigma code paths agree."""
import numpy as np
import pytest

import oracle as O
from paper_2411_07920_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def full():
    from paper_2411_07920_gb300 import swcs
    w = I.workload("so52_e12")
    c = swcs.Context()
    c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    c.apply_ansatz(w.ops[:199], w.theta[:199], w.n_keep)
    k199, a199 = c.get_state()
    c.apply_ansatz(w.ops, w.theta, w.n_keep)
    k, a = c.get_state()
    yield w, c, k199, a199, k, a
    c.close()


def test_last_gate_bit_exact_at_full_size(full):
    import math
    w, c, k199, a199, k, a = full
    assert len(k) == w.n_keep
    th = w.theta[199]
    ko, ao = O.gate(k199, a199, w.ops[199], math.cos(th), math.sin(th), w.n_keep)
    assert np.array_equal(k, ko)
    assert np.array_equal(a, ao)


def test_state_properties_at_full_size(full):
    w, c, _, _, k, a = full
    assert len(np.unique(k)) == len(k)
    pc = np.array([bin(int(x)).count("1") for x in k[::997]])
    assert (pc == w.n_e).all()
    alpha = np.array([bin(int(x) & 0x5555555555555555).count("1") for x in k[::997]])
    assert (alpha == w.n_e // 2).all()
    assert np.all(a != 0.0)
    assert 0.0 < (a * a).sum() <= 1.0 + 1e-12


def test_sigma_and_energy_sampled_at_full_size(full):
    w, c, _, _, k, a = full
    ks, sg = c.get_sigma()
    assert np.array_equal(ks, k)
    rng = np.random.default_rng(0)
    pick = np.concatenate([[int(np.argmax(np.abs(a)))], rng.choice(len(k), 40, replace=False)])
    so = O.sigma_at(w.n_so, w.h, w.g, k, a, k[pick])
    assert np.abs(sg[pick] - so).max() < TOL
    e_int, n2 = c.energy()
    assert abs(e_int - (a @ sg) / (a @ a)) < TOL
    c.pool_gradients()
    e_sw, n2_sw = c.sweep_energy()
    assert abs(e_sw - e_int) < TOL and abs(n2_sw - n2) < 1e-9


def test_pool_gradient_sampled_at_full_size(full):
    """Every operator's support here is >= 4e3 determinants (each orbital pair
    is co-occupied that often), so the oracle's pull form would take minutes
    per operator.  Sampled gradients are pinned by a property that holds at
    any size instead: g_k = dE/dtheta at 0 with U_k appended (untruncated),
    by central differences through the gate kernel and the sigma-int energy
    kernel; and the hashed external-table sweep must agree with the row sweep."""
    w, c, _, _, k, a = full
    g = c.pool_gradients()
    pool = c.pool_ops()
    order = np.argsort(-np.abs(g))
    rng = np.random.default_rng(2)
    picks = list(order[:3]) + list(rng.choice(len(g), 2, replace=False))
    h = 1e-4
    for kk in picks:
        es = []
        for sgn in (1.0, -1.0):
            c.apply_ansatz(w.ops, w.theta, w.n_keep)
            c.apply_gates(pool[kk][None, :], np.array([sgn * h]), 0)
            es.append(c.energy()[0])
        fd = (es[0] - es[1]) / (2 * h)
        assert abs(fd - g[kk]) < 1e-7, (kk, fd, g[kk])
    c.apply_ansatz(w.ops, w.theta, w.n_keep)
    c.set_option("sweep", 1)
    g1 = c.pool_gradients()
    c.set_option("sweep", 0)
    assert np.abs(g1 - g).max() < TOL
