"""ADAPT-VQE (Sec. II.C, Fig. 1) and the BFGS-2 / BFGS-2F bootstrap
procedures (Sec. IV.D), driven through the library.

Host orchestration only: every state, energy, pool gradient (step 4 of
Fig. 1) and parameter gradient (step 7) comes from the library's kernels
(swcs_apply_ansatz, swcs_pool_gradients, swcs_energy_grad).  The host keeps
the operator list, picks the largest |g_k| and runs SciPy's BFGS (the
optimiser of Sec. III) over the parameters.

One iteration: apply the ansatz, sweep the pool (g_k for each operator
appended at the end), stop when ||g|| < eps, else append the operator of
largest |g_k| with parameter 0 and re-optimise:
  "bfgs"    BFGS over all parameters;
  "bfgs2"   BFGS over the new parameter alone (the others frozen), then over all;
  "bfgs2f"  the first half only (the others stay frozen).
With pool="spin" the candidates are the spin-complemented operators of
Sec. III: kappa_k + s kappa_j for each pair the library's
swcs_pool_spin_pairs reports (flip(kappa_k) = s kappa_j), one parameter t
applied as the two gates exp(t kappa_k) exp(s t kappa_j) -- a
self-complementary operator as the one gate exp(2 t kappa_k) -- so its pool
gradient is g_k + s g_j and its parameter gradient the chain-rule sum over
its gates.

Conventions where the paper is silent: |g_k| within a relative 1e-5 of the
largest count as equal (spin-partner operators of a spin-symmetric state
differ only by the optimiser's tolerance) and the first in canonical pool
order wins; an
iteration whose optimisation lowers the energy by less than `stall` is
undone and ends the run (with the state at N_CUT, a new operator at
parameter 0 only reaches determinants the truncation cuts, so its
fixed-projector derivative is zero and the same operator would be chosen
again); a bootstrap stage then continues with the next, larger N_CUT.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import scipy.optimize as opt

from . import swcs


def largest_gradient(g, rel=1e-5):
    """Index of the largest |g_k|; near-ties go to the lowest index."""
    a = np.abs(np.asarray(g))
    return int(np.flatnonzero(a >= a.max() * (1.0 - rel))[0])


@dataclass
class Iteration:
    grad_norm: float
    op_index: int = -1          # -1: converged before choosing
    energy: float = float("nan")
    n_params: int = 0
    energy_grad_calls: int = 0
    n_dets: int = 0
    t_pool_s: float = 0.0       # step 4 (state + pool sweep)
    t_vqe_s: float = 0.0        # step 7 (BFGS over swcs_energy_grad)
    stalled: bool = False


@dataclass
class Adapt:
    ctx: swcs.Context
    n_keep: int
    eps: float = 1e-2
    gtol: float = 1e-6
    ckpt_every: int = 20
    stall: float = 1e-12
    pool_kind: str = "gsd"      # "gsd": every pool operator; "spin": spin-complemented pairs
    theta: np.ndarray = field(default_factory=lambda: np.zeros(0))  # one per chosen candidate
    chosen: list = field(default_factory=list)                      # candidate indices, in order
    history: list = field(default_factory=list)

    def __post_init__(self):
        self.pool = self.ctx.pool_ops()
        P = len(self.pool)
        if self.pool_kind == "spin":
            partner, sign = self.ctx.pool_spin_pairs()
            k = np.arange(P)
            keep = (k < partner) | ((k == partner) & (sign == 1))
            self.unit_k = k[keep]
            self.unit_j = partner[keep]
            self.unit_s = sign[keep].astype(np.float64)
        elif self.pool_kind == "gsd":
            self.unit_k = np.arange(P)
            self.unit_j = np.full(P, -1, np.int64)
            self.unit_s = np.ones(P)
        else:
            raise ValueError(f"unknown pool {self.pool_kind!r}")
        self._calls = 0

    def _expand(self, chosen, theta):
        """Gates of the chosen units: (ops, gate angles, owner unit, factor)."""
        owner, factor, idx = [], [], []
        for i, u in enumerate(chosen):
            k, j, s = int(self.unit_k[u]), int(self.unit_j[u]), float(self.unit_s[u])
            if j < 0:
                idx.append(k); owner.append(i); factor.append(1.0)
            elif j == k:
                idx.append(k); owner.append(i); factor.append(2.0)
            else:
                idx += [k, j]; owner += [i, i]; factor += [1.0, s]
        owner = np.asarray(owner, np.int64)
        factor = np.asarray(factor)
        ops = self.pool[np.asarray(idx, np.int64)] if idx else np.zeros((0, 5), np.uint8)
        return ops, np.asarray(theta)[owner] * factor, owner, factor

    @property
    def ops(self):
        """Gate list of the current ansatz."""
        return self._expand(self.chosen, self.theta)[0]

    def _energy_grad(self, chosen, theta):
        self._calls += 1
        ops, ang, owner, factor = self._expand(chosen, theta)
        e, d = self.ctx.energy_grad(ops, ang, self.n_keep, self.ckpt_every)
        return e, np.bincount(owner, weights=d * factor, minlength=len(theta))

    def _apply(self, chosen, theta):
        ops, ang, _, _ = self._expand(chosen, theta)
        self.ctx.apply_ansatz(ops, ang, self.n_keep)

    def energy(self):
        self._apply(self.chosen, self.theta)
        return self.ctx.energy()[0]

    def pool_gradient(self):
        """Step 4: the gradient of every candidate appended at the end."""
        self._apply(self.chosen, self.theta)
        g = self.ctx.pool_gradients()
        out = g[self.unit_k].copy()
        pair = self.unit_j >= 0
        out[pair] += self.unit_s[pair] * g[self.unit_j[pair]]
        return out

    def _minimize(self, chosen, theta, free):
        """BFGS over theta[free:] with theta[:free] frozen."""
        frozen = theta[:free].copy()

        def fun(x):
            e, d = self._energy_grad(chosen, np.concatenate([frozen, x]))
            return e, d[free:]
        res = opt.minimize(fun, theta[free:], jac=True, method="BFGS", options={"gtol": self.gtol})
        return np.concatenate([frozen, np.asarray(res.x, np.float64)])

    def step(self, optimizer="bfgs"):
        """One ADAPT iteration; False when converged or stalled."""
        t0 = time.perf_counter()
        g = self.pool_gradient()
        e_before = self.ctx.sweep_energy()[0]  # the pool sweep forms sigma, hence E, too
        t1 = time.perf_counter()
        it = Iteration(grad_norm=float(np.linalg.norm(g)), n_params=len(self.theta))
        it.t_pool_s = t1 - t0
        if it.grad_norm < self.eps:
            it.energy = e_before
            self.history.append(it)
            return False
        k = largest_gradient(g)
        chosen = self.chosen + [k]
        theta = np.append(self.theta, 0.0)
        calls0 = self._calls
        if optimizer in ("bfgs2", "bfgs2f"):
            theta = self._minimize(chosen, theta, len(theta) - 1)
        if optimizer in ("bfgs", "bfgs2"):
            theta = self._minimize(chosen, theta, 0)
        if optimizer not in ("bfgs", "bfgs2", "bfgs2f"):
            raise ValueError(f"unknown optimizer {optimizer!r}")
        self._apply(chosen, theta)
        e_after = self.ctx.energy()[0]
        it.t_vqe_s = time.perf_counter() - t1
        it.energy_grad_calls = self._calls - calls0
        it.op_index = k
        if e_after > e_before - self.stall:
            it.stalled = True
            it.energy = e_before
            self.history.append(it)
            return False
        self.chosen, self.theta = chosen, theta
        it.energy = e_after
        it.n_params = len(theta)
        it.n_dets = self.ctx.state_size()
        self.history.append(it)
        return True

    def run(self, max_iter, optimizer="bfgs"):
        """Iterate until converged, stalled or max_iter; True when converged."""
        for _ in range(max_iter):
            if not self.step(optimizer):
                return not self.history[-1].stalled
        return False


def bootstrap(ctx, schedule, max_iter, eps=1e-2, gtol=1e-6, first="bfgs2", then="bfgs2f", **kw):
    """ADAPT at N_CUT = schedule[0] with `first`, continued on the same ansatz
    at each later N_CUT with `then` (BFGS-2 then BFGS-2F in Sec. IV.D)."""
    a = Adapt(ctx, schedule[0], eps=eps, gtol=gtol, **kw)
    stages = []
    for i, n_keep in enumerate(schedule):
        a.n_keep = int(n_keep)
        conv = a.run(max_iter, first if i == 0 else then)
        stages.append(dict(n_keep=int(n_keep), n_params=len(a.theta), converged=conv,
                           stalled=bool(a.history and a.history[-1].stalled), energy=a.history[-1].energy))
    return a, stages


def vqe(ctx, ops, theta0, n_keep, gtol=1e-6, ckpt_every=20):
    """VQE for a fixed ansatz (Eq. 1), e.g. the MP2-ordered UCCSD of
    ctx.mp2_uccsd(): SciPy BFGS over swcs_energy_grad.  Returns (E, theta, calls)."""
    calls = [0]

    def fun(x):
        calls[0] += 1
        return ctx.energy_grad(ops, x, n_keep, ckpt_every)
    res = opt.minimize(fun, np.asarray(theta0, np.float64), jac=True, method="BFGS", options={"gtol": gtol})
    theta = np.asarray(res.x, np.float64)
    ctx.apply_ansatz(ops, theta, n_keep)
    return ctx.energy()[0], theta, calls[0]
