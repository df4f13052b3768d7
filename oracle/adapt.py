"""CPU oracle of the ADAPT-VQE outer loop (Sec. II.C, Fig. 1) and of the
BFGS-2 / BFGS-2F bootstrap procedures (Sec. IV.D) — test infrastructure only.

The loop, step by step as Fig. 1 orders it, on top of the oracle's SWCS:
  step 3  the reference determinant, empty ansatz;
  step 4  the pool gradient: g_k for every generalized single and double
          appended to the end of the current (truncated) ansatz;
  step 5  converged when ||g|| < eps;
  step 6  append the operator with the largest |g_k|, its parameter 0
          (reading: values within a relative 1e-5 of the largest count as
          equal -- spin-partner operators of a spin-symmetric state differ
          only by the optimiser's tolerance -- and the first of them in
          canonical pool order is taken);
  step 7  VQE: BFGS over all parameters, energy and gradient of the
          truncated circuit from the oracle's adjoint.
BFGS-2 replaces step 7 by (1) BFGS over the new parameter alone, the others
frozen at their previous optimum, then (2) BFGS over all of them; BFGS-2F
keeps (1) only.  A bootstrap runs ADAPT with a first N_CUT and continues the
same ansatz with larger N_CUT values, one stage after the other.
An optimisation that lowers E by less than 1e-12 is undone and ends the run
(reading: the same operator would be chosen again).

With pool="spin" the operators are the spin-complemented pairs of Sec. III
(oracle.spin): kappa_k + sign kappa_partner, one parameter t acting as the
gates exp(t kappa_k) exp(sign t kappa_partner) (one gate exp(2 t kappa_k) for
a self-complementary operator); its gradients follow by the chain rule,
g = g_k + sign g_partner.

The optimiser is SciPy's BFGS (the one of Sec. III), used as a library
primitive; its convergence threshold is the gradient norm `gtol` (1e-6 in
Sec. III).

Parity status: pinned by tests/test_adapt_oracle.py — the first iteration
against the 2x2 eigenproblem of the reference and the chosen excitation
(dense Jordan-Wigner Hamiltonian), the BFGS-2 first step against the
closed-form minimum of the exact one-parameter energy, the variational bound
and monotone energies against dense FCI, frozen parameters under BFGS-2F.
"""
from __future__ import annotations

import numpy as np
import scipy.optimize as so

from . import oracle as O
from .spin import spin_units


def _largest(g, rel=1e-5):
    mag = np.abs(np.asarray(g, np.float64))
    top = mag.max()
    for k in range(len(mag)):
        if mag[k] >= top * (1.0 - rel):
            return k
    return int(np.argmax(mag))


class OracleAdapt:
    """ADAPT-VQE state: Hamiltonian, pool, ansatz so far, N_CUT."""

    def __init__(self, n_so, n_e, h, g, n_keep, eps=1e-2, gtol=1e-6, pool="gsd"):
        self.n_so, self.n_e, self.h, self.g = n_so, n_e, h, g
        self.n_keep = n_keep
        self.eps, self.gtol = eps, gtol
        self.pool = O.pool_ops(n_so)
        if pool == "spin":
            self.units = spin_units(self.pool)
        else:
            self.units = [(k, -1, 1) for k in range(len(self.pool))]
        self.chosen = []            # unit indices, in ansatz order
        self.theta = np.zeros(0)    # one parameter per chosen unit
        self.energies = []
        self.grad_norms = []
        self.calls = 0
        self.stalled = False

    def _gates(self, chosen):
        """(ops, owner, factor): gate j applies exp(factor_j theta[owner_j] kappa)."""
        ops, owner, factor = [], [], []
        for i, u in enumerate(chosen):
            k, j, s = self.units[u]
            if j < 0:
                ops.append(self.pool[k]); owner.append(i); factor.append(1.0)
            elif j == k:
                ops.append(self.pool[k]); owner.append(i); factor.append(2.0)
            else:
                ops += [self.pool[k], self.pool[j]]; owner += [i, i]; factor += [1.0, float(s)]
        return np.array(ops, np.uint8).reshape(-1, 5), np.array(owner, np.int64), np.array(factor)

    @property
    def ops(self):
        return self._gates(self.chosen)[0]

    def _eg(self, theta, chosen=None):
        self.calls += 1
        ops, owner, factor = self._gates(self.chosen if chosen is None else chosen)
        e, d = O.energy_grad(self.n_so, self.n_e, self.h, self.g, ops, theta[owner] * factor, self.n_keep)
        dt = np.zeros(len(theta))
        for j in range(len(d)):
            dt[owner[j]] += factor[j] * d[j]
        return e, dt

    def _energy(self, chosen, theta):
        ops, owner, factor = self._gates(chosen)
        keys, amps = O.apply_ansatz(self.n_so, self.n_e, ops, theta[owner] * factor, self.n_keep)
        return O.energy(self.n_so, self.h, self.g, keys, amps)[0]

    def pool_gradient(self):
        """Gradient of every pool unit appended at the end (step 4)."""
        ops, owner, factor = self._gates(self.chosen)
        keys, amps = O.apply_ansatz(self.n_so, self.n_e, ops, self.theta[owner] * factor, self.n_keep)
        g = O.pool_gradients(self.n_so, self.h, self.g, keys, amps)
        out = np.zeros(len(self.units))
        for u, (k, j, s) in enumerate(self.units):
            out[u] = g[k] if j < 0 else g[k] + s * g[j]
        return out

    def _bfgs_all(self, theta, chosen):
        r = so.minimize(lambda t: self._eg(t, chosen), theta, jac=True, method="BFGS",
                        options={"gtol": self.gtol})
        return np.asarray(r.x, np.float64)

    def _bfgs_last(self, theta, chosen):
        head = theta[:-1].copy()

        def f(t):
            e, d = self._eg(np.concatenate([head, t]), chosen)
            return e, d[-1:]
        r = so.minimize(f, theta[-1:], jac=True, method="BFGS", options={"gtol": self.gtol})
        return np.concatenate([head, np.asarray(r.x, np.float64)])

    def iterate(self, mode="bfgs"):
        """One pass of steps 4-7; False once converged (step 5) or stalled."""
        g = self.pool_gradient()
        norm = float(np.sqrt(np.sum(g * g)))
        self.grad_norms.append(norm)
        self.stalled = False
        if norm < self.eps:
            return False
        e_before = self._energy(self.chosen, self.theta)
        u = _largest(g)
        chosen = self.chosen + [u]
        theta = np.concatenate([self.theta, [0.0]])
        if mode in ("bfgs2", "bfgs2f"):
            theta = self._bfgs_last(theta, chosen)
        if mode in ("bfgs", "bfgs2"):
            theta = self._bfgs_all(theta, chosen)
        e_after = self._energy(chosen, theta)
        if not e_after < e_before - 1e-12:
            self.stalled = True
            return False
        self.chosen = chosen
        self.theta = theta
        self.energies.append(e_after)
        return True

    def run(self, max_iter, mode="bfgs"):
        """True when converged (||g|| < eps); False when stalled or out of iterations."""
        for _ in range(max_iter):
            if not self.iterate(mode):
                return not self.stalled
        return False


def bootstrap(n_so, n_e, h, g, schedule, max_iter, eps=1e-2, gtol=1e-6, first="bfgs2", then="bfgs2f",
              pool="gsd"):
    """ADAPT with N_CUT = schedule[0] (optimiser `first`), continued with
    schedule[1:] (optimiser `then`), at most max_iter iterations per stage."""
    a = OracleAdapt(n_so, n_e, h, g, schedule[0], eps, gtol, pool)
    stages = []
    for i, n_keep in enumerate(schedule):
        a.n_keep = n_keep
        conv = a.run(max_iter, first if i == 0 else then)
        stages.append(dict(n_keep=n_keep, n_params=len(a.theta), converged=conv, stalled=a.stalled))
    return a, stages
