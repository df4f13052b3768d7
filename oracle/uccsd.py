"""CPU oracle of the MP2-ordered UCCSD initial guess (Sec. II.A, Eq. 1 with the
operators of Eqs. 2-3) and of the infidelity against a reference state
(Sec. IV.B) — test infrastructure only.

UCCSD ansatz from the reference determinant (spin-orbitals 0 .. n_e - 1
occupied): every S_z-conserving double i<j -> a<b (i, j occupied, a, b
virtual) with its first-order (MP2) amplitude as initial parameter,
  t = <ab||ij> / (e_i + e_j - e_a - e_b),  e_p = h_pp + sum_{k occ} <pk||pk>,
ordered by |t| descending (equal |t| in canonical (i, j, a, b) order), then
every S_z-conserving single i -> a with parameter 0, in canonical order.
Readings: the orbital energies are the diagonal Fock elements of the
reference (the synthetic orbitals are not canonical, so this is the
diagonal Moller-Plesset partitioning); the singles, which have no
first-order double-excitation amplitude, follow the doubles.

Infidelity: 1 - |<a|b>|^2 / (<a|a> <b|b>) of two sparse states.

Parity status: pinned by tests/test_uccsd_oracle.py (amplitudes against the
first-order Rayleigh-Schrodinger coefficients of the dense Jordan-Wigner
Hamiltonian with orbital energies from Koopmans-type dense matrix elements;
overlaps against dense statevectors).
"""
from __future__ import annotations

import numpy as np


def orbital_energies(h, g, n_so, n_e):
    h = np.asarray(h, np.float64).reshape(n_so, n_so)
    g = np.asarray(g, np.float64).reshape(n_so, n_so, n_so, n_so)
    return np.array([h[p, p] + sum(g[p, k, p, k] for k in range(n_e)) for p in range(n_so)])


def mp2_uccsd(h, g, n_so, n_e):
    """(ops [M, 5] uint8, theta [M]) of the MP2-ordered UCCSD ansatz."""
    g = np.asarray(g, np.float64).reshape(n_so, n_so, n_so, n_so)
    eps = orbital_energies(h, g, n_so, n_e)
    occ, vir = range(n_e), range(n_e, n_so)
    doubles = []
    for i in occ:
        for j in occ:
            if j <= i:
                continue
            for a in vir:
                for b in vir:
                    if b <= a or (i % 2) + (j % 2) != (a % 2) + (b % 2):
                        continue
                    t = g[a, b, i, j] / (eps[i] + eps[j] - eps[a] - eps[b])
                    doubles.append(((2, i, j, a, b), t))
    order = sorted(range(len(doubles)), key=lambda q: -abs(doubles[q][1]))  # stable: ties keep canonical order
    ops = [doubles[q][0] for q in order]
    theta = [doubles[q][1] for q in order]
    for i in occ:
        for a in vir:
            if i % 2 == a % 2:
                ops.append((1, i, a, 0, 0))
                theta.append(0.0)
    return np.array(ops, np.uint8).reshape(-1, 5), np.array(theta, np.float64)


def overlap(keys_a, amps_a, keys_b, amps_b):
    """<a|b> of two sparse states (real amplitudes)."""
    b = dict(zip(np.asarray(keys_b, np.uint64).tolist(), np.asarray(amps_b, np.float64).tolist()))
    s = 0.0
    for k, v in zip(np.asarray(keys_a, np.uint64).tolist(), np.asarray(amps_a, np.float64).tolist()):
        s += v * b.get(k, 0.0)
    return s


def infidelity(keys_a, amps_a, keys_b, amps_b):
    ab = overlap(keys_a, amps_a, keys_b, amps_b)
    aa = float(np.dot(amps_a, amps_a))
    bb = float(np.dot(amps_b, amps_b))
    return 1.0 - ab * ab / (aa * bb)


def vqe(n_so, n_e, h, g, ops, theta0, n_keep, gtol=1e-6):
    """BFGS (SciPy, Sec. III) over the oracle's energy and adjoint gradient for
    a fixed ansatz; returns (E, theta)."""
    import scipy.optimize as so
    from . import oracle as O
    res = so.minimize(lambda x: O.energy_grad(n_so, n_e, h, g, ops, x, n_keep), np.asarray(theta0, np.float64),
                      jac=True, method="BFGS", options={"gtol": gtol})
    keys, amps = O.apply_ansatz(n_so, n_e, ops, res.x, n_keep)
    return O.energy(n_so, h, g, keys, amps)[0], np.asarray(res.x, np.float64)
