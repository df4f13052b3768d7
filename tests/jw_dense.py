"""Dense Jordan-Wigner reference used to pin the oracle (tiny systems only).

Built from Kronecker products of Pauli matrices, independently of the
oracle's bitstring phase code: qubit p is bit p of the basis index and
a_p = I x ... x I x sigma^- x Z x ... x Z (Z on every qubit below p).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_SM = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))  # |0><1|: annihilates an occupied mode
_Z = sp.csr_matrix(np.diag([1.0, -1.0]))
_I = sp.identity(2, format="csr")


def annihilators(n):
    ops = []
    for p in range(n):
        m = sp.identity(1, format="csr")
        # kron(A, B): A acts on the more significant bits.  Build from qubit n-1 down to 0.
        for q in range(n - 1, -1, -1):
            f = _I if q > p else (_SM if q == p else _Z)
            m = sp.kron(m, f, format="csr")
        ops.append(m)
    return ops


def tau_matrix(a, op):
    kind, i0, i1, i2, i3 = [int(x) for x in op]
    ad = lambda p: a[p].T.tocsr()
    if kind == 1:
        return (ad(i1) @ a[i0]).tocsr()
    return (ad(i2) @ ad(i3) @ a[i1] @ a[i0]).tocsr()


def kappa_matrix(a, op):
    t = tau_matrix(a, op)
    return (t - t.T).tocsr()


def sector(n, n_e, sz0=True):
    out = []
    for occ in itertools.combinations(range(n), n_e):
        if sz0 and sum(1 for p in occ if p % 2 == 0) * 2 != n_e:
            continue
        out.append(sum(1 << p for p in occ))
    return np.array(sorted(out), dtype=np.int64)


def hamiltonian_sector(n, h, g, basis):
    """Dense H on the given basis from second quantisation with JW matrices:
    H = sum h_pq a+_p a_q + sum_{p<q, r<s} <pq||rs> (a_q a_p)^+ (a_s a_r)."""
    a = annihilators(n)
    dim = 1 << n
    P = sp.csr_matrix((np.ones(len(basis)), (basis, np.arange(len(basis)))), shape=(dim, len(basis)))
    aP = [(a[p] @ P).tocsr() for p in range(n)]
    H = np.zeros((len(basis), len(basis)))
    for p in range(n):
        for q in range(n):
            if h[p, q] != 0.0:
                H += h[p, q] * (aP[p].T @ aP[q]).toarray()
    pairs = [(p, q) for p in range(n) for q in range(p + 1, n)]
    n_e = bin(int(basis[0])).count("1")
    rows = np.array([d for d in range(dim) if bin(d).count("1") == n_e - 2], dtype=np.int64)
    B = [(a[q] @ aP[p]).tocsr()[rows, :] for (p, q) in pairs]   # a_q a_p restricted to the basis
    G = np.array([[g[p, q, r, s] for (r, s) in pairs] for (p, q) in pairs])
    stack = np.stack([b.toarray() for b in B])  # (npairs, n_e-2 sector, nb)
    C = np.tensordot(G, stack, axes=([1], [0]))  # C[P] = sum_R G[P,R] B_R
    H += np.einsum("pdi,pdj->ij", stack, C)
    return H


def statevector(n, n_e, ops, theta):
    a = annihilators(n)
    psi = np.zeros(1 << n)
    psi[(1 << n_e) - 1] = 1.0
    for op, th in zip(ops, theta):
        psi = spla.expm_multiply(th * kappa_matrix(a, op), psi)
    return psi
