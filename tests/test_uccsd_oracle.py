"""Pins for the MP2-ordered UCCSD guess and the infidelity of the oracle, each
independent of its formulas:

* orbital energies from Koopmans-type energy differences of single
  determinants in the N-1 and N+1 electron spaces of the dense Jordan-Wigner
  Hamiltonian;
* every double's initial parameter equals the first-order Rayleigh-Schrodinger
  coefficient <D|H|HF> / (E0_HF - E0_D) of the dense Hamiltonian (with the
  operator's phase on the reference), the doubles in descending |t|, then the
  singles at zero;
* overlaps and infidelities against dense statevectors and the FCI ground state.
"""
import numpy as np

import jw_dense as J
import oracle as O
from oracle.uccsd import infidelity, mp2_uccsd, orbital_energies, overlap
from paper_2411_07920_gb300 import inputs as I


_SECTORS = {}


def _diag(n, h, g, n_e, det):
    """<det|H|det> in the n_e-electron space (any S_z), dense Jordan-Wigner."""
    key = (n, n_e, id(h))
    if key not in _SECTORS:
        basis = J.sector(n, n_e, sz0=False)
        _SECTORS[key] = ({int(b): i for i, b in enumerate(basis)}, J.hamiltonian_sector(n, h, g, basis))
    idx, H = _SECTORS[key]
    return H[idx[det], idx[det]]


def test_orbital_energies_are_koopmans_differences():
    w = I.workload("so12_e4")
    n, ne = w.n_so, w.n_e
    hf = (1 << ne) - 1
    e_hf = _diag(n, w.h, w.g, ne, hf)
    eps = orbital_energies(w.h, w.g, n, ne)
    for p in range(n):
        if p < ne:
            ref = e_hf - _diag(n, w.h, w.g, ne - 1, hf & ~(1 << p))
        else:
            ref = _diag(n, w.h, w.g, ne + 1, hf | (1 << p)) - e_hf
        assert abs(eps[p] - ref) < 1e-12


def test_mp2_amplitudes_are_first_order_coefficients():
    w = I.workload("so12_e4")
    n, ne = w.n_so, w.n_e
    hf = (1 << ne) - 1
    basis = J.sector(n, ne)
    H = J.hamiltonian_sector(n, w.h, w.g, basis)
    idx = {int(b): k for k, b in enumerate(basis)}
    e_hf = H[idx[hf], idx[hf]]
    eps = np.array([e_hf - _diag(n, w.h, w.g, ne - 1, hf & ~(1 << p)) if p < ne else
                    _diag(n, w.h, w.g, ne + 1, hf | (1 << p)) - e_hf for p in range(n)])
    ops, theta = mp2_uccsd(w.h, w.g, n, ne)
    aops = J.annihilators(n)
    v = np.zeros(1 << n)
    v[hf] = 1.0
    nd = int(np.count_nonzero(ops[:, 0] == 2))
    assert np.all(ops[:nd, 0] == 2) and np.all(ops[nd:, 0] == 1) and np.all(theta[nd:] == 0.0)
    assert np.all(np.diff(np.abs(theta[:nd])) <= 0)
    assert nd == len(I.hf_excitation_list(n, ne)) - (len(ops) - nd)
    e0 = lambda d: sum(eps[p] for p in range(n) if d >> p & 1)
    for op, t in zip(ops[:nd], theta[:nd]):
        tv = J.tau_matrix(aops, op) @ v
        d = int(np.flatnonzero(tv)[0])
        c1 = H[idx[d], idx[hf]] / (e0(hf) - e0(d))
        assert abs(t - tv[d] * c1) < 1e-12 * max(1.0, abs(c1))


def test_overlap_and_infidelity_against_dense_vectors():
    w = I.workload("so12_e4")
    n, ne = w.n_so, w.n_e
    basis = J.sector(n, ne)
    H = J.hamiltonian_sector(n, w.h, w.g, basis)
    _, vecs = np.linalg.eigh(H)
    fci = np.zeros(1 << n)
    fci[basis] = vecs[:, 0]
    k, a = O.apply_ansatz(n, ne, w.ops, w.theta, 0)
    psi = np.zeros(1 << n)
    psi[k.astype(np.int64)] = a
    kf = np.flatnonzero(fci).astype(np.uint64)
    af = fci[kf.astype(np.int64)]
    assert abs(overlap(k, a, kf, af) - psi @ fci) < 1e-14
    ref = 1.0 - (psi @ fci) ** 2 / ((psi @ psi) * (fci @ fci))
    assert abs(infidelity(k, a, kf, af) - ref) < 1e-13
    assert abs(infidelity(k, a, k, 3.0 * a)) < 1e-15
    assert infidelity(k[:1], a[:1], k[1:2], a[1:2]) == 1.0


def test_uccsd_vqe_is_bounded_by_fci_and_the_reference():
    w = I.workload("so12_e4")
    n, ne = w.n_so, w.n_e
    from oracle.uccsd import vqe
    ops, theta = mp2_uccsd(w.h, w.g, n, ne)
    e, th = vqe(n, ne, w.h, w.g, ops, theta, 0)
    basis = J.sector(n, ne)
    H = J.hamiltonian_sector(n, w.h, w.g, basis)
    efci = np.linalg.eigvalsh(H)[0]
    hf = (1 << ne) - 1
    e_hf = H[int(np.flatnonzero(basis == hf)[0]), int(np.flatnonzero(basis == hf)[0])]
    k, a = O.apply_ansatz(n, ne, ops, theta, 0)
    e_mp2 = O.energy(n, w.h, w.g, k, a)[0]
    assert efci - 1e-12 <= e <= e_mp2 + 1e-12 and e < e_hf
    _, d = O.energy_grad(n, ne, w.h, w.g, ops, th, 0)
    assert np.abs(d).max() < 1e-5
