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
    ops: np.ndarray = field(default_factory=lambda: np.zeros((0, 5), np.uint8))
    theta: np.ndarray = field(default_factory=lambda: np.zeros(0))
    chosen: list = field(default_factory=list)
    history: list = field(default_factory=list)

    def __post_init__(self):
        self.pool = self.ctx.pool_ops()
        self._calls = 0

    def _energy_grad(self, ops, theta):
        self._calls += 1
        return self.ctx.energy_grad(ops, theta, self.n_keep, self.ckpt_every)

    def energy(self):
        self.ctx.apply_ansatz(self.ops, self.theta, self.n_keep)
        return self.ctx.energy()[0]

    def pool_gradient(self):
        self.ctx.apply_ansatz(self.ops, self.theta, self.n_keep)
        return self.ctx.pool_gradients()

    def _minimize(self, ops, theta, free):
        """BFGS over theta[free:] with theta[:free] frozen."""
        frozen = theta[:free].copy()

        def fun(x):
            e, d = self._energy_grad(ops, np.concatenate([frozen, x]))
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
        ops = np.concatenate([self.ops, self.pool[k:k + 1]])
        theta = np.append(self.theta, 0.0)
        calls0 = self._calls
        if optimizer in ("bfgs2", "bfgs2f"):
            theta = self._minimize(ops, theta, len(theta) - 1)
        if optimizer in ("bfgs", "bfgs2"):
            theta = self._minimize(ops, theta, 0)
        if optimizer not in ("bfgs", "bfgs2", "bfgs2f"):
            raise ValueError(f"unknown optimizer {optimizer!r}")
        self.ctx.apply_ansatz(ops, theta, self.n_keep)
        e_after = self.ctx.energy()[0]
        it.t_vqe_s = time.perf_counter() - t1
        it.energy_grad_calls = self._calls - calls0
        it.op_index = k
        if e_after > e_before - self.stall:
            it.stalled = True
            it.energy = e_before
            self.history.append(it)
            return False
        self.ops, self.theta = ops, theta
        self.chosen.append(k)
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
