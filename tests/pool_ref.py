"""Host-side references for the tests: pool operators applied to single
determinants, their supports, and the pool gradient or one shard of it
contracted from sigma_E values (Sec. II.C: g_k = 2<psi|H A_k|psi>/<psi|psi>,
A_k = tau_k - tau_k^dag).  Plain Python on integers; sigma comes from the
caller (the oracle's pull form, or the library's swcs_sigma_at)."""
import math

import numpy as np


def tau(op, d):
    """(sign, tau d) or None for the pool operator op = (kind, i0..i3) on the integer d:
    tau = a+_{i1} a_{i0} (kind 1) or a+_{i2} a+_{i3} a_{i1} a_{i0} (kind 2), applied right to left."""
    kind, i0, i1, i2, i3 = (int(x) for x in op)
    ann, cre = ([i0], [i1]) if kind == 1 else ([i0, i1], [i2, i3])
    par = 0
    for p in ann:  # a_{i0} first, then a_{i1}
        if not (d >> p) & 1:
            return None
        par ^= bin(d & ((1 << p) - 1)).count("1") & 1
        d ^= 1 << p
    for p in reversed(cre):  # then a+_{i3}, a+_{i2} (a+_{i1} for singles)
        if (d >> p) & 1:
            return None
        par ^= bin(d & ((1 << p) - 1)).count("1") & 1
        d |= 1 << p
    return (-1.0 if par else 1.0), d


def tau_dag(op, d):
    kind, i0, i1, i2, i3 = (int(x) for x in op)
    inv = np.array([kind, i1, i0, 0, 0]) if kind == 1 else np.array([kind, i2, i3, i0, i1])
    return tau(inv, d)


def support(op, k):
    """Indices of the determinants on which tau or tau^dag of the pool operator op acts."""
    kind, i0, i1, i2, i3 = (int(x) for x in op)
    lo = np.uint64((1 << i0) | (1 << i1) if kind == 2 else 1 << i0)
    hi = np.uint64((1 << i2) | (1 << i3) if kind == 2 else 1 << i1)
    up = ((k & lo) == lo) & ((k & hi) == 0)
    dn = ((k & hi) == hi) & ((k & lo) == 0)
    return np.nonzero(up | dn)[0]


def alpha_rank(d, n_so):
    """Colex rank of the alpha string of d: sum over its occupied spatial orbitals p_i
    (ascending) of C(p_i, i + 1)."""
    r, i = 0, 0
    for p in range(n_so // 2):
        if (d >> (2 * p)) & 1:
            i += 1
            r += math.comb(p, i)
    return r


def shard_partial(n_so, pool, keys, amps, sigma_at, shard, n_shards):
    """One shard of the pool sweep: the unscaled gradient sum over the pairs (D, E)
    whose E has alpha_rank(E) = shard (mod n_shards), the energy numerator
    sum c_D sigma_D over the D it owns, and <psi|psi>.  sigma_at(list of E) -> sigma."""
    terms = []  # (k, coefficient, E)
    for kk, op in enumerate(pool):
        for i in support(op, keys):
            d = int(keys[i])
            for f, sgn in ((tau, 1.0), (tau_dag, -1.0)):
                t = f(op, d)
                if t is not None and alpha_rank(t[1], n_so) % n_shards == shard:
                    terms.append((kk, sgn * t[0] * float(amps[i]), t[1]))
    own = [i for i, d in enumerate(keys) if alpha_rank(int(d), n_so) % n_shards == shard]
    dets = [e for _, _, e in terms] + [int(keys[i]) for i in own]
    sig = sigma_at(np.array(dets, np.uint64)) if dets else np.zeros(0)
    graw = np.zeros(len(pool))
    for (kk, cf, _), s in zip(terms, sig[:len(terms)]):
        graw[kk] += cf * s
    num = float(np.dot(amps[own], sig[len(terms):])) if own else 0.0
    return graw, num, float(amps @ amps)
