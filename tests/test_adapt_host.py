"""CPU checks of the ADAPT host loop (paper_2411_07920_gb300.adapt: Sec. II.C,
Fig. 1; BFGS-2 / BFGS-2F and the bootstrap of Sec. IV.D).

The loop only orchestrates library calls, so its host logic -- candidate
units of the spin-complemented pool, chain rule over a unit's gates, the
near-tie rule, BFGS with frozen parameters, the stall rule, the bootstrap
stages -- is run here against a stand-in context whose state, energies and
gradients come from the oracle, and compared with the oracle's own,
independently written loop.  The stand-in exists only in this test; on a
GPU the same loop runs over the CUDA library (tests/test_gpu_adapt.py)."""
import numpy as np
import pytest

import oracle as O
from oracle.adapt import OracleAdapt, bootstrap as oracle_bootstrap
from oracle.spin import spin_pairs
from paper_2411_07920_gb300 import inputs as I


@pytest.fixture(scope="module")
def adapt():
    from paper_2411_07920_gb300 import _build
    _build.build()
    from paper_2411_07920_gb300 import adapt as mod
    return mod


class OracleContext:
    """The Context methods the ADAPT loop calls, computed by the oracle."""

    def __init__(self, w):
        self.w = w
        self.keys = np.array([(1 << w.n_e) - 1], np.uint64)
        self.amps = np.ones(1)
        self.last_sweep_energy = None

    def pool_ops(self):
        return O.pool_ops(self.w.n_so)

    def pool_spin_pairs(self):
        return spin_pairs(O.pool_ops(self.w.n_so))

    def apply_ansatz(self, ops, theta, n_keep):
        self.keys, self.amps = O.apply_ansatz(self.w.n_so, self.w.n_e, ops, theta, n_keep)

    def energy(self):
        return O.energy(self.w.n_so, self.w.h, self.w.g, self.keys, self.amps)

    def pool_gradients(self):
        self.last_sweep_energy = self.energy()
        return O.pool_gradients(self.w.n_so, self.w.h, self.w.g, self.keys, self.amps)

    def sweep_energy(self):
        return self.last_sweep_energy

    def energy_grad(self, ops, theta, n_keep, ckpt_every):
        return O.energy_grad(self.w.n_so, self.w.n_e, self.w.h, self.w.g, ops, theta, n_keep)

    def state_size(self):
        return len(self.keys)


def _accepted(a):
    return [it.energy for it in a.history if it.op_index >= 0 and not it.stalled]


def test_largest_gradient_near_ties_go_to_the_lowest_index(adapt):
    assert adapt.largest_gradient([0.1, -0.5, 0.3]) == 1
    assert adapt.largest_gradient([0.3, -0.5 * (1 - 5e-6), 0.5]) == 1   # within 1e-5 of the largest
    assert adapt.largest_gradient([0.3, -0.5 * (1 - 2e-5), 0.5]) == 2   # outside it
    assert adapt.largest_gradient([0.0, 0.0]) == 0


@pytest.mark.parametrize("pool,n_keep,mode,iters", [
    ("gsd", 0, "bfgs", 8), ("gsd", 20, "bfgs2", 6), ("spin", 0, "bfgs2f", 6), ("spin", 20, "bfgs", 6)])
def test_host_loop_matches_the_oracle_loop(adapt, pool, n_keep, mode, iters):
    w = I.small_case(12, 4, 1, 1)
    ref = OracleAdapt(w.n_so, w.n_e, w.h, w.g, n_keep, eps=1e-3, pool=pool)
    conv_ref = ref.run(iters, mode)
    a = adapt.Adapt(OracleContext(w), n_keep, eps=1e-3, pool_kind=pool)
    conv = a.run(iters, mode)
    # the candidate units are the same in both loops
    if pool == "spin":
        units = [(int(k), int(j), int(s)) for k, j, s in zip(a.unit_k, a.unit_j, a.unit_s)]
        assert units == [(int(k), int(j), int(s)) for k, j, s in ref.units]
    assert conv == conv_ref
    assert a.chosen == ref.chosen
    assert bool(a.history[-1].stalled) == bool(ref.stalled)
    assert np.abs(np.array(_accepted(a)) - np.array(ref.energies)).max() < 1e-12
    assert np.abs(a.theta - ref.theta).max() < 1e-9
    assert np.abs(np.array([it.grad_norm for it in a.history]) - np.array(ref.grad_norms)).max() < 1e-12
    assert np.array_equal(a.ops, ref.ops)


def test_bfgs2f_leaves_earlier_parameters_frozen(adapt):
    w = I.small_case(12, 4, 1, 1)
    a = adapt.Adapt(OracleContext(w), 0, eps=1e-3)
    for _ in range(3):
        before = a.theta.copy()
        if not a.step("bfgs2f"):
            break
        assert np.array_equal(a.theta[:len(before)], before)


def test_unknown_pool_and_optimizer_are_rejected(adapt):
    w = I.small_case(12, 4, 1, 1)
    with pytest.raises(ValueError):
        adapt.Adapt(OracleContext(w), 0, pool_kind="qeb")
    a = adapt.Adapt(OracleContext(w), 0, eps=1e-3)
    with pytest.raises(ValueError):
        a.step("adam")


def test_host_bootstrap_matches_the_oracle_bootstrap(adapt):
    w = I.small_case(12, 4, 1, 3)
    sched = [6, 18, 60]
    ref, st_ref = oracle_bootstrap(w.n_so, w.n_e, w.h, w.g, sched, 4, eps=1e-3)
    a, st = adapt.bootstrap(OracleContext(w), sched, 4, eps=1e-3)
    for key in ("n_keep", "n_params", "converged", "stalled"):
        assert [s[key] for s in st] == [s[key] for s in st_ref]
    assert a.chosen == ref.chosen
    assert np.abs(np.array(_accepted(a)) - np.array(ref.energies)).max() < 1e-12


def test_autograd_wrapper_carries_the_adjoint():
    """SwcsEnergy (paper_2411_07920_gb300.autograd) returns E and hands the
    stored dE/dtheta to torch's backward, scaled by the incoming gradient."""
    import torch
    from paper_2411_07920_gb300.autograd import energy
    w = I.small_case(12, 4, 6, 1)
    ctx = OracleContext(w)
    e_ref, d_ref = O.energy_grad(w.n_so, w.n_e, w.h, w.g, w.ops, w.theta, 0)
    theta = torch.tensor(w.theta, dtype=torch.float64, requires_grad=True)
    e = energy(theta, ctx, w.ops, 0)
    assert abs(e.item() - e_ref) < 1e-14
    (g,) = torch.autograd.grad(3.0 * e, theta)
    assert np.abs(g.numpy() - 3.0 * d_ref).max() < 1e-14
    # untruncated, the adjoint is the derivative of the forward: torch's finite-difference check
    assert torch.autograd.gradcheck(lambda t: energy(t, ctx, w.ops, 0), (theta,), eps=1e-6, atol=1e-7)
