"""Spin complements of the generalized singles and doubles pool (Sec. III:
spin-complemented operators for closed-shell molecules) — test
infrastructure only.

Each pool operator is written as its product of creation and annihilation
operators (tau = a+_q a_p for a single, a+_r a+_s a_q a_p for a double), every
spin-orbital is flipped (2i + s -> 2i + 1 - s), and the string is brought to
the pool's order — creators ascending, annihilators descending — by adjacent
transpositions, each a factor -1.  The result is a pool string, or the
adjoint of one (then the generator kappa = tau - tau^dag changes sign).

Parity status: pinned by tests/test_spin_oracle.py (gradients of a state
symmetrised under the spin flip satisfy g_k = sign_k g_partner(k) for every
operator; commuting pairs reproduce the exponential of the summed generator
on the dense statevector).
"""
from __future__ import annotations

import numpy as np


def _word(op):
    kind, i0, i1, i2, i3 = (int(x) for x in op)
    if kind == 1:
        return [(True, i1), (False, i0)]
    return [(True, i2), (True, i3), (False, i1), (False, i0)]


def _ordered(word):
    """Creators first in ascending index, then annihilators in descending
    index; returns (tuple, sign of the permutation)."""
    w = list(word)
    sign = 1

    def rank(t):
        return (0, t[1]) if t[0] else (1, -t[1])
    done = False
    while not done:
        done = True
        for i in range(len(w) - 1):
            if rank(w[i]) > rank(w[i + 1]):
                w[i], w[i + 1] = w[i + 1], w[i]
                sign = -sign
                done = False
    return tuple(w), sign


def _dagger(word):
    return [(not c, i) for c, i in reversed(word)]


def spin_pairs(pool):
    """(partner, sign) with flip(kappa_k) = sign[k] * kappa_{partner[k]}."""
    table = {}
    for k, op in enumerate(pool):
        w, s = _ordered(_word(op))
        assert s == 1
        table[w] = k
    partner = np.zeros(len(pool), np.int64)
    sign = np.zeros(len(pool), np.int8)
    for k, op in enumerate(pool):
        flipped, s = _ordered([(c, i ^ 1) for c, i in _word(op)])
        if flipped in table:
            partner[k], sign[k] = table[flipped], s
        else:
            adj, s2 = _ordered(_dagger(list(flipped)))
            # tau_flip = s * W, W = s2 * tau_j^dag  =>  kappa_flip = -s * s2 * kappa_j
            partner[k], sign[k] = table[adj], -s * s2
    return partner, sign


def spin_units(pool):
    """Spin-complemented operators as (k, partner, sign) with k <= partner;
    a self-complementary operator with sign -1 has a zero generator and is left out."""
    partner, sign = spin_pairs(pool)
    units = []
    for k in range(len(pool)):
        j = int(partner[k])
        if k < j or (k == j and sign[k] == 1):
            units.append((k, j, int(sign[k])))
    return units
