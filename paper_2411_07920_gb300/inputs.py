"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module only draws random numbers and lays out index lists.  It holds none
of the solver's arithmetic (no gate, phase, Slater-Condon rule, truncation or
gradient), so that the oracle and the CUDA library can both be fed from it
without sharing any code of the method.

The paper's molecules (Sec. III, Tables I-III: STO-3G 10-18 spin-orbitals,
BeH2 / H2O cc-pVDZ 46, C2 cc-pVDZ 52) need PySCF integrals, which are not
available; these generators stand in with the same orbital counts.

Conventions (shared by every consumer):
  * spin-orbital p = 2*spatial + spin, spin 0 = alpha, 1 = beta;
  * h[p, q]      one-electron integrals in the spin-orbital basis;
  * g[p, q, r, s] = <pq||rs> = <pq|rs> - <pq|sr>, physicists' notation,
    with <PQ|RS> = (pr|qs) delta(sP, sR) delta(sQ, sS);
  * an operator is 5 bytes (kind, i0, i1, i2, i3):
      kind 1  tau = a+_{i1} a_{i0}
      kind 2  tau = a+_{i2} a+_{i3} a_{i1} a_{i0}
    and the gate is exp(theta (tau - tau^dagger))  (Eqs. 2-3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

OP_DTYPE = np.uint8  # ops arrays have shape (n_ops, 5)


# --------------------------------------------------------------------------
# Hamiltonian
# --------------------------------------------------------------------------
def spatial_integrals(n_spatial: int, seed: int):
    """Spatial one- and two-electron integrals.

    h: symmetric, diagonal = sorted U(-2, 1) orbital energies, off-diagonal
    N(0, 0.05).  (pq|rs): one draw exp(-|p-q|-|r-s|) * U(0, 0.5) per
    8-fold-symmetric canonical quadruple, copied to all 8 images.
    """
    rng = np.random.default_rng(seed)
    n = n_spatial
    eps = np.sort(rng.uniform(-2.0, 1.0, size=n))
    h = np.zeros((n, n))
    off = rng.normal(0.0, 0.05, size=(n, n))
    for p in range(n):
        for q in range(p):
            h[p, q] = h[q, p] = off[p, q]
        h[p, p] = eps[p]
    eri = np.zeros((n, n, n, n))
    for p in range(n):
        for q in range(p + 1):
            pq = p * (p + 1) // 2 + q
            for r in range(n):
                for s in range(r + 1):
                    rs = r * (r + 1) // 2 + s
                    if rs > pq:
                        continue
                    v = math.exp(-abs(p - q) - abs(r - s)) * rng.uniform(0.0, 0.5)
                    for (a, b, c, d) in ((p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                                         (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)):
                        eri[a, b, c, d] = v
    return h, eri, eps


def spin_orbital_integrals(h_sp: np.ndarray, eri_sp: np.ndarray):
    """Spin-orbital h[p,q] and antisymmetrised <pq||rs> (interleaved spin)."""
    n = h_sp.shape[0]
    N = 2 * n
    sp = np.arange(N) // 2
    sg = np.arange(N) % 2
    h = np.where(sg[:, None] == sg[None, :], h_sp[sp[:, None], sp[None, :]], 0.0)
    # <PQ|RS> = (pr|qs) d(sP,sR) d(sQ,sS)
    P = np.arange(N)[:, None, None, None]
    Q = np.arange(N)[None, :, None, None]
    R = np.arange(N)[None, None, :, None]
    S = np.arange(N)[None, None, None, :]
    direct = eri_sp[sp[P], sp[R], sp[Q], sp[S]] * ((sg[P] == sg[R]) & (sg[Q] == sg[S]))
    exch = eri_sp[sp[P], sp[S], sp[Q], sp[R]] * ((sg[P] == sg[S]) & (sg[Q] == sg[R]))
    g = direct - exch
    return np.ascontiguousarray(h), np.ascontiguousarray(g)


def hamiltonian(n_so: int, seed: int):
    """(h, g, eps) for n_so spin-orbitals; g[p,q,r,s] = <pq||rs>."""
    if n_so % 2:
        raise ValueError("n_so must be even (two spins per spatial orbital)")
    h_sp, eri_sp, eps = spatial_integrals(n_so // 2, seed)
    h, g = spin_orbital_integrals(h_sp, eri_sp)
    return h, g, eps


# --------------------------------------------------------------------------
# Operator lists used as ansatz inputs
# --------------------------------------------------------------------------
def hf_excitation_list(n_so: int, n_e: int) -> np.ndarray:
    """S_z-conserving occupied->virtual singles and doubles relative to the
    reference determinant (bits 0..n_e-1 set), as (n, 5) uint8 rows.

    Order: singles by (i, a), then doubles by ((i, j), (a, b)), i<j, a<b.
    """
    occ = list(range(n_e))
    vir = list(range(n_e, n_so))
    rows = []
    for i in occ:
        for a in vir:
            if i % 2 == a % 2:
                rows.append((1, i, a, 0, 0))
    for ii, i in enumerate(occ):
        for j in occ[ii + 1:]:
            for ia, a in enumerate(vir):
                for b in vir[ia + 1:]:
                    if (i % 2) + (j % 2) == (a % 2) + (b % 2):
                        rows.append((2, i, j, a, b))
    return np.asarray(rows, dtype=OP_DTYPE).reshape(-1, 5)


def draw_ansatz(n_so: int, n_e: int, n_ops: int, seed: int, theta: str):
    """n_ops operators drawn uniformly without replacement from the
    occupied->virtual list (kept in draw order) and their angles."""
    rng = np.random.default_rng(seed)
    pool = hf_excitation_list(n_so, n_e)
    n_ops = min(n_ops, len(pool))
    sel = rng.choice(len(pool), size=n_ops, replace=False)
    ops = np.ascontiguousarray(pool[sel])
    if theta == "uniform0.1":
        th = rng.uniform(-0.1, 0.1, size=n_ops)
    elif theta == "normal0.05":
        th = rng.normal(0.0, 0.05, size=n_ops)
    else:
        raise ValueError(theta)
    return ops, np.ascontiguousarray(th, dtype=np.float64)


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    n_so: int
    n_e: int
    h: np.ndarray
    g: np.ndarray
    eps: np.ndarray
    ops: np.ndarray
    theta: np.ndarray
    n_keep: int
    ckpt_every: int = 20
    meta: dict = field(default_factory=dict)


_SPECS = {
    # 12 spin-orbitals / 4 electrons (FCI dimension 225), 10 gates, no truncation
    "so12_e4": dict(n_so=12, n_e=4, seed=1, n_ops=10, theta="uniform0.1", n_keep=0),
    # 28 / 8, 60 gates, top-1e5 after every gate
    "so28_e8": dict(n_so=28, n_e=8, seed=2, n_ops=60, theta="normal0.05", n_keep=100_000),
    # 52 / 12, 200 gates, top-1e6 after every gate (gradient, sweep and adjoint workload)
    "so52_e12": dict(n_so=52, n_e=12, seed=3, n_ops=200, theta="normal0.05", n_keep=1_000_000),
}


def workload(name: str, n_keep: int | None = None, n_ops: int | None = None) -> Workload:
    s = dict(_SPECS[name])
    if n_keep is not None:
        s["n_keep"] = n_keep
    if n_ops is not None:
        s["n_ops"] = n_ops
    h, g, eps = hamiltonian(s["n_so"], s["seed"])
    ops, th = draw_ansatz(s["n_so"], s["n_e"], s["n_ops"], s["seed"], s["theta"])
    return Workload(name=name, n_so=s["n_so"], n_e=s["n_e"], h=h, g=g, eps=eps, ops=ops,
                    theta=th, n_keep=s["n_keep"], meta=dict(seed=s["seed"]))


def small_case(n_so: int, n_e: int, n_ops: int, seed: int, n_keep: int = 0,
               theta: str = "normal0.05") -> Workload:
    """Ad-hoc workload of the same recipe (used for edge-case tests)."""
    h, g, eps = hamiltonian(n_so, seed)
    ops, th = draw_ansatz(n_so, n_e, n_ops, seed, theta)
    if theta == "normal0.05":
        th = th * 4.0  # larger angles spread the amplitudes over more determinants
    return Workload(name=f"so{n_so}_e{n_e}_s{seed}", n_so=n_so, n_e=n_e, h=h, g=g, eps=eps,
                    ops=ops, theta=np.ascontiguousarray(th), n_keep=n_keep, meta=dict(seed=seed))


def batch_specs(n_inst: int = 64, seed0: int = 100):
    """Uneven instances: n_so in U{16..40} even, n_e in U{4..12} even,
    gates in U{20..150}, n_keep log-uniform in [1e3, 1e5].  Each instance has
    its own seed (seed0 + i) for integrals and ansatz."""
    out = []
    for i in range(n_inst):
        rng = np.random.default_rng(seed0 + i)
        n_so = int(rng.integers(8, 21)) * 2
        n_e = int(rng.integers(2, 7)) * 2
        n_e = min(n_e, n_so - 2)
        n_gates = int(rng.integers(20, 151))
        n_keep = int(round(10 ** rng.uniform(3.0, 5.0)))
        out.append(dict(n_so=n_so, n_e=n_e, n_gates=n_gates, n_keep=n_keep, seed=seed0 + i))
    return out


def batch_instance(spec: dict) -> Workload:
    h, g, eps = hamiltonian(spec["n_so"], spec["seed"])
    ops, th = draw_ansatz(spec["n_so"], spec["n_e"], spec["n_gates"], spec["seed"], "normal0.05")
    return Workload(name=f"inst{spec['seed']}", n_so=spec["n_so"], n_e=spec["n_e"], h=h, g=g,
                    eps=eps, ops=ops, theta=th, n_keep=spec["n_keep"], meta=dict(spec))
