"""Parity at the benchmark's full size (52 spin-orbitals, 12 electrons,
200 gates, N = 1e6) in the launch configuration bench.py times, on outputs
the oracle can compute one at a time:
  * the last gate with its truncation, bit-exact, from the GPU's state after
    199 gates (the oracle's own full run takes minutes);
  * sigma_D on sampled determinants (oracle pulls each from its connections);
  * sigma_E on sampled external determinants, read out of the pool sweep's own
    rows, against the oracle's pull; the samples include determinants whose
    only connections to the state are of one excitation class (alpha-alpha
    doubles, beta singles, ...), so each of the sweep's loops is pinned alone;
  * the pool gradient of sampled operators contracted on the host from those
    sweep-row sigmas, against the sweep's own gradient;
  * the 200-parameter adjoint against central differences of the energy with
    every truncation held as the fixed projector the derivative is defined
    with (gates replayed untruncated, then projected on the kept sets);
  * properties at any size: N kept determinants, particle number, S_z, the
    energies of the two sigma code paths agree."""
import numpy as np
import pytest

import oracle as O
from paper_2411_07920_gb300 import inputs as I

import pool_ref as R

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


# ---------------------------------------------------------------- external sigma at full size
_POP16 = np.array([bin(i).count("1") for i in range(1 << 16)], np.int8)


def _popc32(x):
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(x)
    return _POP16[x & np.uint32(0xFFFF)] + _POP16[x >> np.uint32(16)]


def _spin_strings(k, n_so):
    """Per determinant its alpha and beta strings as packed uint32 (bit p = spatial orbital p)."""
    k = np.asarray(k, np.uint64)
    xa = np.zeros(k.shape, np.uint32)
    xb = np.zeros(k.shape, np.uint32)
    for p in range(n_so // 2):
        xa |= ((k >> np.uint64(2 * p)) & np.uint64(1)).astype(np.uint32) << np.uint32(p)
        xb |= ((k >> np.uint64(2 * p + 1)) & np.uint64(1)).astype(np.uint32) << np.uint32(p)
    return xa, xb


class _Connections:
    """Counts, per excitation class, of the state determinants connected to a
    determinant e: alpha distance on the distinct alpha strings first, beta
    distance only on the determinants of the alpha groups within reach."""
    KINDS = {"diag": (0, 0), "a": (2, 0), "b": (0, 2), "aa": (4, 0), "bb": (0, 4), "ab": (2, 2)}

    def __init__(self, k, n_so):
        self.n_so = n_so
        ka, kb = _spin_strings(k, n_so)
        order = np.argsort(ka, kind="stable")
        self.ka, self.kb = ka[order], kb[order]
        self.ua, self.start, self.count = np.unique(self.ka, return_index=True, return_counts=True)

    def __call__(self, e):
        ea, eb = _spin_strings(np.array([e], np.uint64), self.n_so)
        da = _popc32(self.ua ^ ea[0])
        near = np.nonzero(da <= 4)[0]
        idx = np.concatenate([np.arange(s, s + c) for s, c in zip(self.start[near], self.count[near])]) \
            if len(near) else np.zeros(0, np.int64)
        pa = np.repeat(da[near], self.count[near])
        pb = _popc32(self.kb[idx] ^ eb[0])
        return {t: int(((pa == u) & (pb == v)).sum()) for t, (u, v) in self.KINDS.items()}


def _excite(d, spin, n_exc, rng, n_so):
    occ = [p for p in range(spin, n_so, 2) if (d >> p) & 1]
    vir = [p for p in range(spin, n_so, 2) if not (d >> p) & 1]
    for p in list(rng.choice(occ, n_exc, replace=False)) + list(rng.choice(vir, n_exc, replace=False)):
        d ^= 1 << int(p)
    return d


def test_external_sigma_sampled_at_full_size(full):
    """sigma_E read from the pool sweep's rows (swcs_sigma_at) against the
    oracle's pull form, on >= 50 external determinants of every class."""
    w, c, _, _, k, a = full
    c.apply_ansatz(w.ops, w.theta, w.n_keep)
    rng = np.random.default_rng(11)
    in_state = set(int(x) for x in k[rng.choice(len(k), 200000, replace=False)])
    big = k[np.argsort(-np.abs(a))[:20000]]
    conn = _Connections(k, w.n_so)
    excitations = {"aa": [(0, 2)], "b": [(1, 1)], "a": [(0, 1)], "bb": [(1, 2)], "ab": [(0, 1), (1, 1)]}
    picked, only = [], {}
    for name, ex in excitations.items():
        found, mixed = [], []
        for _ in range(3000):
            d = int(big[rng.integers(len(big))]) if rng.random() < 0.2 else int(k[rng.integers(len(k))])
            e = d
            for spin, ne in ex:
                e = _excite(e, spin, ne, rng, w.n_so)
            if e in in_state:
                continue
            cl = conn(e)
            if cl["diag"]:
                continue
            nz = {t for t, v in cl.items() if v}
            if nz == {name}:
                found.append(e)
            elif len(mixed) < 6:
                mixed.append(e)
            if len(found) >= 6:
                break
        only[name] = len(found)
        picked += found + mixed[: max(0, 10 - len(found))]
    # determinants with a single class of connections: every loop of the sweep alone
    assert all(v >= 3 for v in only.values()), only
    picked += [int(x) for x in k[rng.choice(len(k), 10, replace=False)]]  # and members of the state
    at = np.array(picked, np.uint64)
    assert len(at) >= 50
    got = c.sigma_at(at)
    want = O.sigma_at(w.n_so, w.h, w.g, k, a, at)
    assert np.abs(got - want).max() < TOL, np.abs(got - want).max()
    assert np.abs(want).max() > 1e-6  # the samples carry real contributions


def test_pool_gradient_from_sweep_sigma_at_full_size(full):
    """g_k = 2/<psi|psi> sum_D c_D (s sigma(tau_k D) - s' sigma(tau_k^dag D)),
    contracted on the host from the sweep rows' sigma at every needed E, for
    sampled operators of small support; equals the sweep's own g_k."""
    w, c, _, _, k, a = full
    c.apply_ansatz(w.ops, w.theta, w.n_keep)
    g = c.pool_gradients()
    pool = c.pool_ops()
    n2 = float(a @ a)
    rng = np.random.default_rng(12)
    cand = rng.choice(len(pool), 400, replace=False)
    sizes = [len(R.support(pool[kk], k)) for kk in cand]
    order = np.argsort(sizes)
    picks = [int(cand[i]) for i in order if sizes[i] > 0][:3]
    for kk in picks:
        terms, dets = [], []
        supp = R.support(pool[kk], k)
        for d, cd in zip(k[supp], a[supp]):
            for f, sgn in ((R.tau, 1.0), (R.tau_dag, -1.0)):
                t = f(pool[kk], int(d))
                if t is not None:
                    terms.append(sgn * t[0] * cd)
                    dets.append(t[1])
        sig = c.sigma_at(np.array(dets, np.uint64))
        gk = 2.0 * float(np.dot(terms, sig)) / n2
        assert abs(gk - g[kk]) < TOL, (kk, gk, g[kk])


def test_adjoint_finite_differences_at_full_size(full):
    """The 200-parameter adjoint (checkpoints every 20 gates) against central
    differences of the energy with every truncation held as the fixed
    projector the derivative is defined with: from the state before gate g,
    each later gate is applied untruncated and the result projected on the
    unperturbed run's kept set of that gate.  (The plain truncated energy is
    not smooth at this size: amplitudes tied at the cut, such as spin-flip
    partners, change places under any perturbation.)  With h = 0 the
    projected replay reproduces the truncated run's energy."""
    w, c, _, _, k_end, _ = full
    e0, d = c.energy_grad(w.ops, w.theta, w.n_keep, 20)
    M = len(w.ops)
    h = 1e-5
    for g in (M - 1, M - 4, M - 12):
        c.apply_ansatz(w.ops[:g], w.theta[:g], w.n_keep)
        k_in, a_in = c.get_state()
        kept = []
        for m in range(g, M):
            c.apply_ansatz(w.ops[:m + 1], w.theta[:m + 1], w.n_keep)
            kept.append(c.get_state()[0])
        es = []
        for step in (0.0, h, -h):
            c.set_state(k_in, a_in)
            for m in range(g, M):
                th = w.theta[m] + (step if m == g else 0.0)
                c.apply_gates(w.ops[m:m + 1], np.array([th]), 0)
                k, a = c.get_state()
                keep = np.isin(k, kept[m - g], assume_unique=True)
                c.set_state(k[keep], a[keep])
            es.append(c.energy()[0])
        assert abs(es[0] - e0) < TOL, (g, es[0], e0)
        fd = (es[1] - es[2]) / (2 * h)
        assert abs(fd - d[g]) < 1e-7, (g, fd, d[g])
    c.apply_ansatz(w.ops, w.theta, w.n_keep)
    assert np.array_equal(c.get_state()[0], k_end)
