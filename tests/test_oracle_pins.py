"""Pins for the CPU oracle: each check is independent of the oracle's own code.

* dense Jordan-Wigner matrices (Kronecker products of Pauli matrices) and
  scipy's expm_multiply for the gate sequence of Eq. 1-3;
* the dense Hamiltonian in the particle sector, its FCI ground state and the
  variational bound;
* closed forms: HF energy, one gate on HF (2x2 block), pool gradient at HF,
  GSD pool size, FCI dimension;
* invariants: norm, particle number, S_z, Hermiticity;
* brute force: truncation by lexicographic sort, pool gradient by forming
  A_k psi explicitly, central finite differences for the adjoint.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as O
from paper_2411_07920_gb300 import inputs as I

import jw_dense as J

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def c1():
    w = I.workload("so12_e4")
    basis = J.sector(w.n_so, w.n_e)
    H = J.hamiltonian_sector(w.n_so, w.h, w.g, basis)
    return w, basis, H


def _dense(keys, amps, n):
    v = np.zeros(1 << n)
    v[np.asarray(keys, dtype=np.int64)] = amps
    return v


# ---------------------------------------------------------------- sizes
def test_fci_dimension_and_pool_size_closed_forms():
    # FCI dimension of 12 spin-orbitals / 4 electrons at S_z = 0: C(6,2)^2 = 225
    assert len(J.sector(12, 4)) == math.comb(6, 2) ** 2 == 225
    for n_so in (8, 12, 28, 52):
        m = n_so // 2
        closed = 2 * math.comb(m, 2) + 6 * math.comb(m, 4) + (m * (m - 1)) ** 2 // 2
        assert O.pool_ops(n_so).shape[0] == closed
    golden = dict(l.split()[:2] for l in open(os.path.join(GOLD, "pool_sizes.txt")) if l[0].isdigit())
    for n_so, cnt in golden.items():
        assert O.pool_ops(int(n_so)).shape[0] == int(cnt)


def test_pool_ops_are_canonical_and_sz_conserving():
    ops = O.pool_ops(12)
    keys = []
    for kind, p, q, r, s in ops:
        if kind == 1:
            assert p < q and p % 2 == q % 2
            keys.append((0, p, q, 0, 0))
        else:
            assert p < q and r < s and (p, q) < (r, s)
            assert len({p, q, r, s}) == 4
            assert sorted((p % 2, q % 2)) == sorted((r % 2, s % 2))
            keys.append((1, p, q, r, s))
    assert keys == sorted(keys) and len(set(keys)) == len(keys)


# ---------------------------------------------------------------- Hamiltonian
def test_hamiltonian_matches_dense_jordan_wigner(c1):
    w, basis, H = c1
    Ho = np.array([[O.h_element(w.n_so, w.h, w.g, int(e), int(d)) for d in basis] for e in basis])
    assert np.abs(H - H.T).max() == 0.0
    assert np.abs(Ho - Ho.T).max() < 1e-14          # Hermiticity (real symmetric)
    assert np.abs(Ho - H).max() < 1e-13


def test_hf_energy_closed_form(c1):
    w, basis, H = c1
    occ = list(range(w.n_e))
    e_hf = sum(w.h[i, i] for i in occ) + 0.5 * sum(w.g[i, j, i, j] for i in occ for j in occ)
    e, n2 = O.energy(w.n_so, w.h, w.g, np.array([(1 << w.n_e) - 1], np.uint64), np.array([1.0]))
    assert n2 == 1.0
    assert abs(e - e_hf) < 1e-13


# ---------------------------------------------------------------- gates
def test_untruncated_circuit_matches_statevector(c1):
    w, basis, H = c1
    psi = J.statevector(w.n_so, w.n_e, w.ops, w.theta)
    k, a = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 0)
    assert np.abs(_dense(k, a, w.n_so) - psi).max() < 1e-14
    # variational bound against FCI
    e, n2 = O.energy(w.n_so, w.h, w.g, k, a)
    assert abs(n2 - 1.0) < 1e-14
    e_fci = np.linalg.eigvalsh(H)[0]
    assert e >= e_fci - 1e-12
    assert abs(e - psi[basis] @ H @ psi[basis]) < 1e-13


@pytest.mark.parametrize("n_so,n_e,seed", [(8, 2, 11), (12, 6, 12), (16, 4, 13)])
def test_larger_angle_circuits_match_statevector(n_so, n_e, seed):
    w = I.small_case(n_so, n_e, 12, seed)
    psi = J.statevector(w.n_so, w.n_e, w.ops, w.theta)
    k, a = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 0)
    assert np.abs(_dense(k, a, w.n_so) - psi).max() < 1e-13
    # invariants: particle number, S_z, norm
    for d in k:
        d = int(d)
        assert bin(d).count("1") == n_e
        assert sum((d >> p) & 1 for p in range(0, n_so, 2)) == n_e // 2
    assert abs((a * a).sum() - 1.0) < 1e-13


def test_one_gate_closed_form(c1):
    w, basis, H = c1
    hf = (1 << w.n_e) - 1
    for op in I.hf_excitation_list(w.n_so, w.n_e)[::7]:
        a = J.annihilators(w.n_so)
        t = J.tau_matrix(a, op)
        v = np.zeros(1 << w.n_so)
        v[hf] = 1.0
        tv = t @ v
        d = int(np.flatnonzero(tv)[0])
        s = tv[d]
        idx = {int(b): i for i, b in enumerate(basis)}
        e_hf, e_d, h_x = H[idx[hf], idx[hf]], H[idx[d], idx[d]], H[idx[hf], idx[d]]
        for th in (0.3, -1.1):
            k, amps = O.apply_ansatz(w.n_so, w.n_e, op[None, :], np.array([th]), 0)
            e, _ = O.energy(w.n_so, w.h, w.g, k, amps)
            closed = math.cos(th) ** 2 * e_hf + math.sin(th) ** 2 * e_d + 2 * s * math.sin(th) * math.cos(th) * h_x
            assert abs(e - closed) < 1e-13


def test_gate_preserves_norm_before_truncation():
    w = I.small_case(16, 6, 20, 21)
    k = np.array([(1 << 6) - 1], np.uint64)
    a = np.array([1.0])
    for op, th in zip(w.ops, w.theta):
        k2, a2 = O.gate(k, a, op, math.cos(th), math.sin(th), 0)
        assert abs((a2 * a2).sum() - (a * a).sum()) < 1e-14 * max(1, len(a))
        k, a = k2, a2


# ---------------------------------------------------------------- truncation
def _lex_top(keys, amps, n_keep):
    nz = amps != 0.0
    keys, amps = keys[nz], amps[nz]
    if n_keep <= 0 or len(keys) <= n_keep:
        sel = np.arange(len(keys))
    else:
        sel = np.lexsort((keys, -np.abs(amps)))[:n_keep]
    order = np.argsort(keys[sel])
    return keys[sel][order], amps[sel][order]


@pytest.mark.parametrize("seed", range(6))
def test_truncation_matches_lexicographic_sort(seed):
    rng = np.random.default_rng(seed)
    n = 2000
    keys = rng.choice(1 << 40, size=n, replace=False).astype(np.uint64)
    amps = rng.normal(size=n)
    # many exact ties in |c| (both signs) and some exact zeros
    amps[rng.integers(0, n, 400)] = 0.125
    amps[rng.integers(0, n, 300)] = -0.125
    amps[rng.integers(0, n, 50)] = 0.0
    for n_keep in (1, 7, 150, 999, 1500, 5000, 0):
        k, a = O.truncate(keys, amps, n_keep)
        k2, a2 = _lex_top(keys, amps, n_keep)
        assert np.array_equal(k, k2) and np.array_equal(a, a2)


def test_truncated_circuit_matches_statevector_with_sort_truncation():
    """Dense statevector with top-N after every gate (ties by key), vs oracle."""
    w = I.small_case(12, 4, 14, 31)
    n_keep = 20
    a_ops = J.annihilators(w.n_so)
    psi = np.zeros(1 << w.n_so)
    psi[(1 << w.n_e) - 1] = 1.0
    for op, th in zip(w.ops, w.theta):
        psi = spla.expm_multiply(th * J.kappa_matrix(a_ops, op), psi)
        idx = np.flatnonzero(psi).astype(np.uint64)
        kk, aa = _lex_top(idx, psi[idx.astype(np.int64)], n_keep)
        psi = _dense(kk, aa, w.n_so)
    k, a = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_keep)
    assert np.abs(_dense(k, a, w.n_so) - psi).max() < 1e-13
    assert len(k) == n_keep


# ---------------------------------------------------------------- pool gradient
def test_pool_gradient_matches_dense_commutator(c1):
    w, basis, H = c1
    k, a = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 0)
    g = O.pool_gradients(w.n_so, w.h, w.g, k, a)
    psi = _dense(k, a, w.n_so)
    pool = O.pool_ops(w.n_so)
    aops = J.annihilators(w.n_so)
    # dense H on the whole 4-electron space (A_k psi may leave S_z = 0? no: pool conserves S_z)
    idx = {int(b): i for i, b in enumerate(basis)}
    for kk in range(0, len(pool), 3):
        chi = J.kappa_matrix(aops, pool[kk]) @ psi
        ref = 2.0 * (psi[basis] @ H @ chi[basis]) / (psi @ psi)
        assert np.abs(chi).sum() == pytest.approx(np.abs(chi[basis]).sum())
        assert abs(g[kk] - ref) < 1e-12


def test_pool_gradient_brute_force_and_subset(c1):
    w, basis, H = c1
    wk = I.small_case(12, 4, 12, 41)
    k, a = O.apply_ansatz(wk.n_so, wk.n_e, wk.ops, wk.theta, 9)
    a = a * 1.7  # unnormalised state: the Rayleigh quotient normalisation must appear
    g = O.pool_gradients(wk.n_so, wk.h, wk.g, k, a)
    gb = O.pool_gradients_brute(wk.n_so, wk.h, wk.g, k, a)
    assert np.abs(g - gb).max() < 1e-13
    sub = np.array([3, 100, 569, 0], np.int64)
    gs = O.pool_gradients(wk.n_so, wk.h, wk.g, k, a, subset=sub)
    assert np.array_equal(gs[sub], g[sub])
    assert np.isnan(np.delete(gs, sub)).all()


def test_pool_gradient_finite_difference():
    """g_k = dE/dtheta at theta=0 for U_k appended after the ansatz (ADAPT step 4)."""
    w = I.small_case(12, 4, 8, 51)
    k, a = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 0)
    g = O.pool_gradients(w.n_so, w.h, w.g, k, a)
    pool = O.pool_ops(w.n_so)
    hstep = 1e-5
    for kk in range(0, len(pool), 37):
        ep = O.energy(w.n_so, w.h, w.g, *O.gate(k, a, pool[kk], math.cos(hstep), math.sin(hstep)))[0]
        em = O.energy(w.n_so, w.h, w.g, *O.gate(k, a, pool[kk], math.cos(-hstep), math.sin(-hstep)))[0]
        assert abs((ep - em) / (2 * hstep) - g[kk]) < 1e-8


def test_pool_gradient_at_hf_closed_form(c1):
    w, basis, H = c1
    hf = (1 << w.n_e) - 1
    g = O.pool_gradients(w.n_so, w.h, w.g, np.array([hf], np.uint64), np.array([1.0]))
    pool = O.pool_ops(w.n_so)
    aops = J.annihilators(w.n_so)
    idx = {int(b): i for i, b in enumerate(basis)}
    v = np.zeros(1 << w.n_so)
    v[hf] = 1.0
    nonzero = 0
    for kk, op in enumerate(pool):
        t = J.tau_matrix(aops, op)
        up, dn = t @ v, t.T @ v
        if up.any():
            d = int(np.flatnonzero(up)[0])
            ref = 2 * up[d] * H[idx[hf], idx[d]]
        elif dn.any():
            d = int(np.flatnonzero(dn)[0])
            ref = -2 * dn[d] * H[idx[hf], idx[d]]
        else:
            ref = 0.0
        nonzero += ref != 0.0
        assert abs(g[kk] - ref) < 1e-13
    assert nonzero > 50


# ---------------------------------------------------------------- adjoint
@pytest.mark.parametrize("zeros", [(), (3, 9), tuple(range(10))])
def test_adjoint_untruncated_matches_dense_derivative(c1, zeros):
    """Also at theta_g = 0 (a new ADAPT parameter), where the gate's partner
    determinants have exactly zero amplitude but a nonzero derivative."""
    w, basis, H = c1
    theta = w.theta.copy()
    theta[list(zeros)] = 0.0
    e, d = O.energy_grad(w.n_so, w.n_e, w.h, w.g, w.ops, theta, 0)
    aops = J.annihilators(w.n_so)
    K = [J.kappa_matrix(aops, op) for op in w.ops]
    psis = [np.zeros(1 << w.n_so)]
    psis[0][(1 << w.n_e) - 1] = 1.0
    for kk, th in zip(K, theta):
        psis.append(spla.expm_multiply(th * kk, psis[-1]))
    Hfull = np.zeros((1 << w.n_so, 1 << w.n_so))
    Hfull[np.ix_(basis, basis)] = H
    lam = Hfull @ psis[-1]
    assert abs(e - psis[-1] @ lam) < 1e-13
    for g in range(len(w.ops) - 1, -1, -1):
        # d psi_M / d theta_g = U_M..U_{g+1} kappa_g psi_g
        dpsi = K[g] @ psis[g + 1]
        for j in range(g + 1, len(w.ops)):
            dpsi = spla.expm_multiply(theta[j] * K[j], dpsi)
        assert abs(2 * lam @ dpsi - d[g]) < 1e-12


@pytest.mark.parametrize("n_keep", [6, 15])
def test_adjoint_truncated_matches_finite_differences(n_keep):
    w = I.small_case(12, 4, 12, 61)
    e, d = O.energy_grad(w.n_so, w.n_e, w.h, w.g, w.ops, w.theta, n_keep)
    M = len(w.ops)

    def kept_sets(theta):
        return [O.apply_ansatz(w.n_so, w.n_e, w.ops[:m], theta[:m], n_keep)[0] for m in range(1, M + 1)]

    sets0 = kept_sets(w.theta)
    hstep = 1e-5
    checked = 0
    for g in range(M):
        tp, tm = w.theta.copy(), w.theta.copy()
        tp[g] += hstep
        tm[g] -= hstep
        same = all(np.array_equal(x, y) for x, y in zip(kept_sets(tp), sets0)) and \
            all(np.array_equal(x, y) for x, y in zip(kept_sets(tm), sets0))
        if not same:
            continue  # a kept set moved under +-h: the fixed-projector derivative does not apply
        kp, ap = O.apply_ansatz(w.n_so, w.n_e, w.ops, tp, n_keep)
        km, am = O.apply_ansatz(w.n_so, w.n_e, w.ops, tm, n_keep)
        fd = (O.energy(w.n_so, w.h, w.g, kp, ap)[0] - O.energy(w.n_so, w.h, w.g, km, am)[0]) / (2 * hstep)
        assert abs(fd - d[g]) < 1e-7
        checked += 1
    assert checked >= len(w.ops) // 2


def test_pull_routes_match_push_routes():
    """sigma pulled at single determinants and the pull-form pool gradient
    against the push-form sigma (internal energy route) and pool gradient."""
    w = I.small_case(12, 4, 20, 81, n_keep=60)
    k, a = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 60)
    sig = O.sigma_internal(w.n_so, w.h, w.g, k, a)
    assert np.abs(O.sigma_at(w.n_so, w.h, w.g, k, a, k) - sig).max() < 1e-13
    g = O.pool_gradients(w.n_so, w.h, w.g, k, a)
    sub = np.arange(0, len(g), 7, dtype=np.int64)
    gp = O.pool_gradients_pull(w.n_so, w.h, w.g, k, a, sub)
    assert np.abs(gp - g[sub]).max() < 1e-13
    # sigma outside the state equals the dense H psi there
    basis = J.sector(w.n_so, w.n_e)
    H = J.hamiltonian_sector(w.n_so, w.h, w.g, basis)
    psi = np.zeros(len(basis))
    idx = {int(b): i for i, b in enumerate(basis)}
    for kk, aa in zip(k, a):
        psi[idx[int(kk)]] = aa
    hp = H @ psi
    pick = basis[::5].astype(np.uint64)
    assert np.abs(O.sigma_at(w.n_so, w.h, w.g, k, a, pick) - hp[::5]).max() < 1e-12


# ---------------------------------------------------------------- magnitude truncation
@pytest.mark.parametrize("eps,n_keep", [(2e-3, 0), (2e-3, 25), (2e-2, 0)])
def test_magnitude_truncated_circuit_matches_statevector(eps, n_keep):
    """Sec. II.B's magnitude criterion: after every gate the dense statevector
    (expm_multiply of Eq. 2) loses every |c| < eps, then keeps the top n_keep."""
    w = I.small_case(12, 4, 14, 33)
    a_ops = J.annihilators(w.n_so)
    psi = np.zeros(1 << w.n_so)
    psi[(1 << w.n_e) - 1] = 1.0
    dropped = 0
    for op, th in zip(w.ops, w.theta):
        psi = spla.expm_multiply(th * J.kappa_matrix(a_ops, op), psi)
        idx = np.flatnonzero(np.abs(psi) >= eps).astype(np.uint64)
        dropped += int(np.count_nonzero(np.abs(psi) > 1e-12)) - len(idx)
        kk, aa = _lex_top(idx, psi[idx.astype(np.int64)], n_keep)
        psi = _dense(kk, aa, w.n_so)
    k, a = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_keep, eps=eps)
    assert dropped > 0  # the criterion acted
    assert np.abs(_dense(k, a, w.n_so) - psi).max() < 1e-13
    assert np.abs(a).min() >= eps


def test_magnitude_truncation_acts_after_every_gate():
    """The same single excitation twice: exp(t2 k) exp(t1 k) = exp((t1+t2) k)
    without truncation; with eps between |sin t1| and |cos t1| the excited
    determinant is dropped after the first gate, so the second gate starts
    again from the reference alone (amplitudes cos t1 cos t2, +-cos t1 sin t2)."""
    n_so, n_e = 8, 2
    op = np.array([1, 0, 2, 0, 0], np.uint8)  # tau = a+_2 a_0
    t1, t2 = 0.05, 0.7
    ops = np.stack([op, op])
    k0, a0 = O.apply_ansatz(n_so, n_e, ops, np.array([t1, t2]), 0)
    assert np.allclose(sorted(np.abs(a0)), sorted([abs(math.cos(t1 + t2)), abs(math.sin(t1 + t2))]), atol=1e-15)
    k, a = O.apply_ansatz(n_so, n_e, ops, np.array([t1, t2]), 0, eps=0.1)
    assert sorted(np.abs(a)) == pytest.approx(sorted([math.cos(t1) * math.sin(t2), math.cos(t1) * math.cos(t2)]),
                                              abs=1e-15)
    assert set(k.tolist()) == {0b11, 0b110}


def test_magnitude_truncated_adjoint_matches_finite_differences():
    w = I.small_case(12, 4, 12, 63)
    eps = 5e-3
    e, d = O.energy_grad(w.n_so, w.n_e, w.h, w.g, w.ops, w.theta, 0, eps=eps)
    M = len(w.ops)

    def kept_sets(theta):
        return [O.apply_ansatz(w.n_so, w.n_e, w.ops[:m], theta[:m], 0, eps=eps)[0] for m in range(1, M + 1)]

    sets0 = kept_sets(w.theta)
    hstep = 1e-5
    checked = 0
    for g in range(M):
        tp, tm = w.theta.copy(), w.theta.copy()
        tp[g] += hstep
        tm[g] -= hstep
        if not (all(np.array_equal(x, y) for x, y in zip(kept_sets(tp), sets0)) and
                all(np.array_equal(x, y) for x, y in zip(kept_sets(tm), sets0))):
            continue
        kp, ap = O.apply_ansatz(w.n_so, w.n_e, w.ops, tp, 0, eps=eps)
        km, am = O.apply_ansatz(w.n_so, w.n_e, w.ops, tm, 0, eps=eps)
        fd = (O.energy(w.n_so, w.h, w.g, kp, ap)[0] - O.energy(w.n_so, w.h, w.g, km, am)[0]) / (2 * hstep)
        assert abs(fd - d[g]) < 1e-7
        checked += 1
    assert checked >= M // 2
    # the criterion dropped determinants on this circuit
    assert len(O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 0)[0]) > len(sets0[-1])


# ---------------------------------------------------------------- stored values
def _stored(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        if line.startswith("#") or not line.strip():
            continue
        key, *vals = line.split()
        out[key] = vals
    return out


def test_stored_oracle_values_reproduce_and_match_dense_statevector(c1):
    """tests/golden/so12_e4_oracle.txt (written by make_golden.py from the
    oracle alone) is a regression pin: the oracle still reproduces it, and its
    energy, determinant count and largest pool gradients agree with the dense
    Jordan-Wigner statevector of the same circuit (Eqs. 1-3), which shares no
    code with the oracle."""
    w, basis, H = c1
    st = _stored("so12_e4_oracle.txt")
    k, a = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 0)
    e, n2 = O.energy(w.n_so, w.h, w.g, k, a)
    g = O.pool_gradients(w.n_so, w.h, w.g, k, a)
    _, d = O.energy_grad(w.n_so, w.n_e, w.h, w.g, w.ops, w.theta, 0)
    assert int(st["n_det"][0]) == len(k)
    assert abs(float(st["energy"][0]) - e) < 1e-14
    assert abs(float(st["norm2"][0]) - n2) < 1e-14
    assert np.abs(np.array(st["dtheta"], float) - d).max() < 1e-13
    top = {int(t.split(":")[0]): float(t.split(":")[1]) for t in st["pool_top"]}
    assert list(top) == [int(i) for i in np.argsort(-np.abs(g))[:10]]
    for kk, v in top.items():
        assert abs(v - g[kk]) < 1e-13
    # the stored numbers against the dense statevector
    psi = J.statevector(w.n_so, w.n_e, w.ops, w.theta)
    assert int(st["n_det"][0]) == int((np.abs(psi) > 0).sum())
    assert abs(float(st["energy"][0]) - psi[basis] @ H @ psi[basis] / (psi @ psi)) < 1e-13
    aops = J.annihilators(w.n_so)
    pool = O.pool_ops(w.n_so)
    for kk, v in top.items():
        chi = J.kappa_matrix(aops, pool[kk]) @ psi
        assert abs(v - 2.0 * (psi[basis] @ H @ chi[basis]) / (psi @ psi)) < 1e-12
