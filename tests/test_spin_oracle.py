"""Pins for the spin-complemented pool of the oracle (Sec. III), independent
of its string manipulation:

* the spin flip U_F (a+_p -> a+_{F(p)}, F(2i+s) = 2i+1-s) commutes with the
  synthetic Hamiltonian, so on a state symmetrised under U_F the pool
  gradients satisfy g_k = sign_k g_partner(k) for every operator -- a wrong
  partner or sign fails wherever the gradient is nonzero;
* for pairs on disjoint spin-orbitals the two gates with a shared parameter
  equal the exponential of the summed generator (dense statevector);
* the pairing is an involution with a symmetric sign.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import jw_dense as J
import oracle as O
from oracle.spin import spin_pairs, spin_units
from paper_2411_07920_gb300 import inputs as I


def _flip_det(d, n_so):
    """U_F |D> = sign |F(D)>, |D> = a+_{p1} a+_{p2} ... |0> with p1 < p2 < ..."""
    occ = [p for p in range(n_so) if d >> p & 1]
    img = [p ^ 1 for p in occ]
    inv = sum(1 for i in range(len(img)) for j in range(i + 1, len(img)) if img[i] > img[j])
    return sum(1 << p for p in img), (-1) ** inv


def _symmetrised(keys, amps, n_so):
    st = {}
    for k, a in zip(keys.tolist(), amps.tolist()):
        st[k] = st.get(k, 0.0) + a
        f, s = _flip_det(k, n_so)
        st[f] = st.get(f, 0.0) + s * a
    ks = np.array(sorted(st), np.uint64)
    return ks, np.array([st[int(k)] for k in ks])


@pytest.mark.parametrize("n_so,n_e,seed", [(12, 4, 3), (16, 6, 4)])
def test_flip_symmetric_state_has_paired_gradients(n_so, n_e, seed):
    w = I.small_case(n_so, n_e, 12, seed)
    pool = O.pool_ops(n_so)
    partner, sign = spin_pairs(pool)
    assert np.array_equal(partner[partner], np.arange(len(pool)))
    assert np.array_equal(sign[partner], sign)
    for d in range(1 << 10):  # U_F is an involution on determinants
        if bin(d).count("1") == 4:
            f, s = _flip_det(d, 10)
            f2, s2 = _flip_det(f, 10)
            assert f2 == d and s * s2 == 1
    keys, amps = O.apply_ansatz(n_so, n_e, w.ops, w.theta, 0)
    ks, a_s = _symmetrised(keys, amps, n_so)
    g = O.pool_gradients(n_so, w.h, w.g, ks, a_s)
    assert np.count_nonzero(np.abs(g) > 1e-6) > len(pool) // 4
    assert np.abs(g - sign * g[partner]).max() < 1e-12
    # the unsymmetrised state breaks the relation (so the check has teeth)
    g0 = O.pool_gradients(n_so, w.h, w.g, keys, amps)
    assert np.abs(g0 - sign * g0[partner]).max() > 1e-4


def test_commuting_pairs_are_the_exponential_of_the_sum():
    n_so, n_e = 12, 4
    w = I.small_case(n_so, n_e, 6, 7)
    pool = O.pool_ops(n_so)
    units = spin_units(pool)
    a = J.annihilators(n_so)
    psi = J.statevector(n_so, n_e, w.ops, w.theta)
    checked = 0
    rng = np.random.default_rng(0)
    for u in rng.choice(len(units), 60, replace=False):
        k, j, s = units[u]
        if k == j:
            continue
        sk = set(int(x) for x in pool[k][1:3 if pool[k][0] == 1 else 5])
        sj = set(int(x) for x in pool[j][1:3 if pool[j][0] == 1 else 5])
        if sk & sj:
            continue
        t = 0.37
        Kk, Kj = J.kappa_matrix(a, pool[k]), J.kappa_matrix(a, pool[j])
        lhs = spla.expm_multiply(t * (Kk + s * Kj), psi)
        rhs = spla.expm_multiply(s * t * Kj, spla.expm_multiply(t * Kk, psi))
        assert np.abs(lhs - rhs).max() < 1e-13
        kk, aa = O.apply_ansatz(n_so, n_e, np.concatenate([w.ops, pool[[k, j]]]),
                                np.concatenate([w.theta, [t, s * t]]), 0)
        v = np.zeros(1 << n_so)
        v[kk.astype(np.int64)] = aa
        assert np.abs(v - lhs).max() < 1e-13
        checked += 1
    assert checked >= 10
