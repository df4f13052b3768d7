"""CPU checks of the seeded synthetic inputs (paper_2411_07920_gb300.inputs):
the integral symmetries a real molecular Hamiltonian has, S_z conservation,
determinism per seed, and the documented ranges of the ansatz and batch
recipes.  These properties are what the oracle and the CUDA path both assume
of their inputs."""
import math

import numpy as np
import pytest

from paper_2411_07920_gb300 import inputs as I


@pytest.mark.parametrize("n_so,seed", [(4, 0), (12, 1), (16, 7)])
def test_integral_symmetries_and_spin_blocks(n_so, seed):
    h, g, eps = I.hamiltonian(n_so, seed)
    assert h.shape == (n_so, n_so) and g.shape == (n_so,) * 4
    assert np.array_equal(h, h.T)
    spin = np.arange(n_so) % 2
    assert not h[spin[:, None] != spin[None, :]].any()              # h conserves spin
    assert np.array_equal(g, -g.transpose(1, 0, 2, 3))              # <pq||rs> = -<qp||rs>
    assert np.array_equal(g, -g.transpose(0, 1, 3, 2))              # <pq||rs> = -<pq||sr>
    assert np.array_equal(g, g.transpose(2, 3, 0, 1))               # real orbitals: <pq||rs> = <rs||pq>
    P, Q, R, S = np.meshgrid(*(spin,) * 4, indexing="ij")
    assert not g[(P + Q) != (R + S)].any()                          # S_z conserved
    assert np.all(np.diff(eps) >= 0) and eps.min() >= -2.0 and eps.max() <= 1.0
    assert np.array_equal(np.diag(h)[0::2], eps) and np.array_equal(np.diag(h)[1::2], eps)


def test_spatial_integrals_have_the_eightfold_symmetry():
    _, eri, _ = I.spatial_integrals(5, 3)
    for perm in ((1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1)):
        assert np.array_equal(eri, eri.transpose(perm))
    assert (eri >= 0).all() and eri.max() <= 0.5


def test_same_seed_same_inputs_other_seed_other_inputs():
    a, b, c = I.workload("so12_e4"), I.workload("so12_e4"), I.small_case(12, 4, 10, 2)
    assert np.array_equal(a.h, b.h) and np.array_equal(a.g, b.g)
    assert np.array_equal(a.ops, b.ops) and np.array_equal(a.theta, b.theta)
    assert not np.array_equal(a.g, c.g)


@pytest.mark.parametrize("n_so,n_e", [(12, 4), (28, 8), (52, 12)])
def test_reference_excitations_are_sz_conserving_and_complete(n_so, n_e):
    ops = I.hf_excitation_list(n_so, n_e)
    singles, doubles = ops[ops[:, 0] == 1], ops[ops[:, 0] == 2]
    assert len(singles) + len(doubles) == len(ops)
    m, k = n_so // 2, n_e // 2   # spatial orbitals, electrons per spin
    v = m - k
    assert len(singles) == 2 * k * v
    assert len(doubles) == 2 * math.comb(k, 2) * math.comb(v, 2) + (k * v) ** 2
    assert (singles[:, 1] < n_e).all() and (singles[:, 2] >= n_e).all()
    assert (singles[:, 1] % 2 == singles[:, 2] % 2).all()
    i, j, a, b = (doubles[:, c].astype(int) for c in range(1, 5))
    assert (i < j).all() and (a < b).all() and (j < n_e).all() and (a >= n_e).all()
    assert ((i % 2 + j % 2) == (a % 2 + b % 2)).all()
    assert len({tuple(r) for r in ops.tolist()}) == len(ops)


def test_benchmark_ansatz_recipe():
    w = I.workload("so52_e12")
    assert (w.n_so, w.n_e, len(w.ops), w.n_keep) == (52, 12, 200, 1_000_000)
    pool = {tuple(r) for r in I.hf_excitation_list(52, 12).tolist()}
    assert all(tuple(r) in pool for r in w.ops.tolist())
    assert len({tuple(r) for r in w.ops.tolist()}) == 200           # drawn without replacement
    assert abs(w.theta.std() - 0.05) < 0.01 and abs(w.theta.mean()) < 0.015


def test_batch_specs_stay_in_their_documented_ranges():
    specs = I.batch_specs()
    assert len(specs) == 64 and [s["seed"] for s in specs] == list(range(100, 164))
    for s in specs:
        assert 16 <= s["n_so"] <= 40 and s["n_so"] % 2 == 0
        assert 4 <= s["n_e"] <= 12 and s["n_e"] % 2 == 0 and s["n_e"] < s["n_so"]
        assert 20 <= s["n_gates"] <= 150
        assert 1000 <= s["n_keep"] <= 100_000
    assert len({(s["n_so"], s["n_e"]) for s in specs}) > 10            # uneven instances
    w = I.batch_instance(specs[0])
    assert len(w.ops) == min(specs[0]["n_gates"], len(I.hf_excitation_list(w.n_so, w.n_e)))
