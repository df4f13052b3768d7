"""Parity of the CUDA path with the oracle, through the C ABI.

Bit-exact: determinant sets and amplitudes after every gate sequence
(each amplitude is a sum of at most two rounded products, so the result is
independent of the order of work).  Energies and pool gradients: 1e-10
(FP64 atomics reorder the sums).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2411_07920_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def S():
    from paper_2411_07920_gb300 import swcs
    return swcs


def ctx_for(S, w):
    c = S.Context()
    c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    return c


def assert_state_equal(k1, a1, k2, a2):
    assert len(k1) == len(k2)
    assert np.array_equal(k1, k2)
    assert np.array_equal(a1, a2), np.abs(a1 - a2).max()


def test_pool_matches_oracle(S):
    for n_so, n_e in ((12, 4), (28, 8), (52, 12)):
        w = I.small_case(n_so, n_e, 1, 1)
        c = ctx_for(S, w)
        assert np.array_equal(c.pool_ops(), O.pool_ops(n_so))


def test_so12_e4_untruncated(S):
    w = I.workload("so12_e4")
    c = ctx_for(S, w)
    c.apply_ansatz(w.ops, w.theta, 0)
    k, a = c.get_state()
    ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, 0)
    assert_state_equal(k, a, ko, ao)
    e, n2 = c.energy()
    eo, n2o = O.energy(w.n_so, w.h, w.g, ko, ao)
    assert abs(e - eo) < TOL and abs(n2 - n2o) < 1e-14
    g = c.pool_gradients()
    go = O.pool_gradients(w.n_so, w.h, w.g, ko, ao)
    assert np.abs(g - go).max() < TOL


@pytest.mark.parametrize("n_so,n_e,n_ops,seed,n_keep", [
    (12, 4, 30, 101, 17), (16, 6, 40, 102, 150), (20, 6, 50, 103, 1000), (28, 8, 60, 104, 3000),
    (16, 4, 25, 105, 1), (16, 4, 25, 106, 10 ** 6)])
def test_truncated_gate_sequence_bit_exact(S, n_so, n_e, n_ops, seed, n_keep):
    w = I.small_case(n_so, n_e, n_ops, seed, n_keep=n_keep)
    c = ctx_for(S, w)
    c.apply_ansatz(w.ops, w.theta, n_keep)
    k, a = c.get_state()
    ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_keep)
    assert_state_equal(k, a, ko, ao)
    # prefixes: every intermediate state too
    for m in (1, 2, n_ops // 2):
        c.apply_ansatz(w.ops[:m], w.theta[:m], n_keep)
        k, a = c.get_state()
        assert_state_equal(k, a, *O.apply_ansatz(w.n_so, w.n_e, w.ops[:m], w.theta[:m], n_keep))


@pytest.mark.parametrize("n_so,n_e,n_ops,seed,n_keep", [(16, 6, 40, 102, 150), (20, 6, 50, 103, 700),
                                                        (24, 8, 40, 107, 400)])
def test_energy_and_pool_gradient_truncated(S, n_so, n_e, n_ops, seed, n_keep):
    w = I.small_case(n_so, n_e, n_ops, seed, n_keep=n_keep)
    c = ctx_for(S, w)
    c.apply_ansatz(w.ops, w.theta, n_keep)
    ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_keep)
    e, n2 = c.energy()
    eo, n2o = O.energy(w.n_so, w.h, w.g, ko, ao)
    assert abs(e - eo) < TOL
    assert abs(n2 - n2o) < 1e-13
    g = c.pool_gradients()
    go = O.pool_gradients(w.n_so, w.h, w.g, ko, ao)
    assert np.abs(g - go).max() < TOL
    sub = np.array([0, 5, len(go) - 1, len(go) // 2], np.int64)
    gs = c.pool_gradients(subset=sub)
    assert np.abs(gs[sub] - go[sub]).max() < TOL


@pytest.mark.parametrize("sweep,cluster,threads,occ", [(1, 4, 512, 3), (2, 1, 128, 3), (2, 2, 256, 3), (2, 4, 512, 3),
                                                       (2, 8, 512, 2), (2, 1, 512, 2), (2, 2, 512, 3), (2, 2, 512, 1),
                                                       (2, 1, 1024, 1), (2, 2, 1024, 1), (2, 4, 1024, 1)])
@pytest.mark.parametrize("n_so,n_e,n_ops,seed,n_keep", [(16, 6, 40, 102, 150), (24, 8, 40, 107, 400),
                                                        (28, 8, 60, 104, 3000), (12, 4, 10, 1, 0)])
def test_sweep_paths_match_oracle(S, sweep, cluster, threads, occ, n_so, n_e, n_ops, seed, n_keep):
    """Hashed external-sigma sweep and alpha-string row sweep, several launch shapes."""
    w = I.small_case(n_so, n_e, n_ops, seed, n_keep=n_keep)
    c = ctx_for(S, w)
    c.set_option("sweep", sweep)
    c.set_option("cluster", cluster)
    c.set_option("threads", threads)
    c.set_option("row_occupancy", occ)
    c.apply_ansatz(w.ops, w.theta, n_keep)
    ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_keep)
    g = c.pool_gradients()
    go = O.pool_gradients(w.n_so, w.h, w.g, ko, ao)
    assert np.abs(g - go).max() < TOL
    e, n2 = c.sweep_energy()
    eo, n2o = O.energy(w.n_so, w.h, w.g, ko, ao)
    assert abs(e - eo) < TOL and abs(n2 - n2o) < 1e-13


@pytest.mark.parametrize("n_so,n_e,n_ops,seed,n_keep", [(16, 6, 40, 102, 150), (28, 8, 60, 104, 3000),
                                                        (12, 4, 10, 1, 0)])
def test_energy_paths_match_oracle(S, n_so, n_e, n_ops, seed, n_keep):
    """Energy through the alpha-string rows and through the probe kernel."""
    w = I.small_case(n_so, n_e, n_ops, seed, n_keep=n_keep)
    c = ctx_for(S, w)
    c.apply_ansatz(w.ops, w.theta, n_keep)
    eo, n2o = O.energy(w.n_so, w.h, w.g, *O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, n_keep))
    for mode in (1, 2):
        c.set_option("energy", mode)
        e, n2 = c.energy()
        assert abs(e - eo) < TOL and abs(n2 - n2o) < 1e-13


def test_truncation_with_ties_and_zeros(S):
    w = I.small_case(20, 6, 1, 7)
    c = ctx_for(S, w)
    rng = np.random.default_rng(5)
    # random S_z = 0 determinants with 3 alpha + 3 beta electrons
    dets = set()
    while len(dets) < 3000:
        al = rng.choice(10, 3, replace=False)
        be = rng.choice(10, 3, replace=False)
        dets.add(sum(1 << (2 * int(x)) for x in al) + sum(1 << (2 * int(x) + 1) for x in be))
    keys = np.array(sorted(dets), np.uint64)
    amps = rng.normal(size=len(keys))
    amps[rng.integers(0, len(keys), 700)] = 0.03125
    amps[rng.integers(0, len(keys), 500)] = -0.03125
    amps[rng.integers(0, len(keys), 100)] = 0.0
    for n_keep in (1, 13, 800, 1111, 2500, 2999, 5000):
        c.set_state(keys, amps)
        c.truncate(n_keep)
        k, a = c.get_state()
        assert_state_equal(k, a, *O.truncate(keys, amps, n_keep))


def test_gate_on_arbitrary_state(S):
    w = I.small_case(20, 6, 40, 8)
    c = ctx_for(S, w)
    ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops[:20], w.theta[:20], 0)
    for op, th, nk in zip(w.ops[20:30], w.theta[20:30] * 7.0, (0, 5, 50, 0, 300, 17, 0, 2, 1000, 40)):
        c.set_state(ko, ao)
        c.apply_gates(op[None, :], np.array([th]), nk)
        k, a = c.get_state()
        ko2, ao2 = O.gate(ko, ao, op, math.cos(th), math.sin(th), nk)
        assert_state_equal(k, a, ko2, ao2)


def test_edge_cases(S):
    w = I.small_case(12, 4, 5, 9)
    c = ctx_for(S, w)
    # no gates: the reference determinant alone
    c.apply_ansatz(w.ops[:0], w.theta[:0], 10)
    k, a = c.get_state()
    assert k.tolist() == [0b1111] and a.tolist() == [1.0]
    e, n2 = c.energy()
    eo, _ = O.energy(12, w.h, w.g, k, a)
    assert abs(e - eo) < TOL and n2 == 1.0
    # theta = 0: zero amplitudes are dropped
    c.apply_ansatz(w.ops, np.zeros(len(w.ops)), 0)
    k, a = c.get_state()
    assert k.tolist() == [0b1111] and a.tolist() == [1.0]
    # a gate that acts on nothing leaves the state unchanged
    c.apply_gates(np.array([[2, 8, 9, 10, 11]], np.uint8), np.array([0.7]), 0)
    assert c.get_state()[0].tolist() == [0b1111]


def test_invalid_arguments_are_rejected(S):
    w = I.small_case(12, 4, 5, 9)
    c = S.Context()
    with pytest.raises(S.SwcsError):
        c.energy()  # no Hamiltonian
    with pytest.raises(S.SwcsError):
        c.load_hamiltonian(np.zeros((11, 11)), np.zeros(11 ** 4), 11, 4)
    c.load_hamiltonian(w.h, w.g, 12, 4)
    for bad in ([[2, 0, 1, 2, 4]], [[2, 0, 2, 4, 5]], [[1, 0, 3, 0, 0]], [[3, 0, 1, 2, 3]], [[1, 0, 40, 0, 0]]):
        with pytest.raises(S.SwcsError) as ei:
            c.apply_ansatz(np.array(bad, np.uint8), np.array([0.1]), 0)
        assert ei.value.code == -1


def test_device_theta_path_matches_host(S):
    import torch
    w = I.small_case(20, 6, 50, 103, n_keep=700)
    c = ctx_for(S, w)
    c.apply_ansatz(w.ops, w.theta, 700)
    k1, a1 = c.get_state()
    c.apply_ansatz_dev(torch.from_numpy(w.ops.reshape(-1)).cuda(), torch.from_numpy(w.theta).cuda(), 700)
    k2, a2 = c.get_state()
    # device sin/cos may differ from the host libm by an ulp
    assert np.array_equal(k1, k2) or len(set(k1.tolist()) ^ set(k2.tolist())) <= 4
    common = np.intersect1d(k1, k2)
    i1, i2 = np.searchsorted(k1, common), np.searchsorted(k2, common)
    assert np.abs(a1[i1] - a2[i2]).max() < 1e-13
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    c.energy_dev(out)
    e, _ = c.energy()
    assert abs(out[0].item() - e) < 1e-12


def test_so28_e8_full_size(S):
    w = I.workload("so28_e8")
    c = ctx_for(S, w)
    c.apply_ansatz(w.ops, w.theta, w.n_keep)
    k, a = c.get_state()
    ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, w.n_keep)
    assert_state_equal(k, a, ko, ao)
    e, n2 = c.energy()
    # sampled gradients: the oracle on a random subset of operators
    g = c.pool_gradients()
    rng = np.random.default_rng(0)
    sub = np.sort(rng.choice(len(g), 200, replace=False)).astype(np.int64)
    go = O.pool_gradients(w.n_so, w.h, w.g, ko, ao, subset=sub)
    assert np.abs(g[sub] - go[sub]).max() < TOL
    # the energy from the sweep's by-product equals the sigma-int energy (two code paths)
    assert abs(e - O.energy(w.n_so, w.h, w.g, ko, ao)[0]) < TOL
    assert abs(c.sweep_energy()[0] - e) < TOL
    # both sweep paths agree at full size
    c.set_option("sweep", 1)
    g1 = c.pool_gradients()
    assert np.abs(g1 - g).max() < TOL


@pytest.mark.parametrize("n_e,n_keep,sweep", [(4, 300, 0), (6, 200, 0), (4, 300, 1)])
def test_largest_orbital_space(S, n_e, n_keep, sweep):
    """64 spin-orbitals, the largest the bitstrings hold: determinants with bit 63 set, the
    708,784-operator pool, 32-orbital alpha strings in the row sweep (sweep 0) and the hashed
    external table (sweep 1)."""
    w = I.small_case(64, n_e, 24, 140 + n_e, n_keep=n_keep)
    top = np.array([[2, 0, 1, 62, 63], [1, n_e - 1, 63, 0, 0]], np.uint8)
    ops = np.concatenate([w.ops, top])
    theta = np.concatenate([w.theta, [0.4, -0.3]])
    c = ctx_for(S, w)
    c.set_option("sweep", sweep)
    c.apply_ansatz(ops, theta, n_keep)
    k, a = c.get_state()
    ko, ao = O.apply_ansatz(64, n_e, ops, theta, n_keep)
    assert_state_equal(k, a, ko, ao)
    assert (ko >> np.uint64(63)).any()
    e, _ = c.energy()
    assert abs(e - O.energy(64, w.h, w.g, ko, ao)[0]) < TOL
    g = c.pool_gradients()
    go = O.pool_gradients(64, w.h, w.g, ko, ao)
    assert len(go) == 708784
    assert np.abs(g - go).max() < TOL


def test_rows_above_two_million_entries(S):
    """64 spin-orbitals and 14 electrons: beta strings of 7 electrons in 32 orbitals give rows of
    3,365,856 entries, above the 2^21 ranks that the packed beta-single entries hold, so the row sweep
    looks the beta pair up from the strings' orbital lists instead."""
    n_e, n_keep = 14, 120
    assert math.comb(32, 7) > 1 << 21
    w = I.small_case(64, n_e, 24, 140 + n_e, n_keep=n_keep)
    top = np.array([[2, 0, 1, 62, 63], [1, n_e - 1, 63, 0, 0]], np.uint8)
    ops = np.concatenate([w.ops, top])
    theta = np.concatenate([w.theta, [0.4, -0.3]])
    c = ctx_for(S, w)
    c.apply_ansatz(ops, theta, n_keep)
    k, a = c.get_state()
    ko, ao = O.apply_ansatz(64, n_e, ops, theta, n_keep)
    assert_state_equal(k, a, ko, ao)
    e, _ = c.energy()
    assert abs(e - O.energy(64, w.h, w.g, ko, ao)[0]) < TOL
    c.set_option("sweep", 2)
    g = c.pool_gradients()
    assert len(g) == 708784
    rng = np.random.default_rng(1)
    sub = np.sort(rng.choice(len(g), 300, replace=False)).astype(np.int64)
    go = O.pool_gradients(64, w.h, w.g, ko, ao, subset=sub)
    assert np.abs(g[sub] - go[sub]).max() < TOL
    assert abs(c.sweep_energy()[0] - e) < TOL
    c.set_option("sweep", 1)
    assert np.abs(c.pool_gradients() - g).max() < TOL


@pytest.mark.parametrize("n_so,n_e", [(12, 2), (12, 10), (8, 6), (4, 2)])
def test_nearly_empty_and_nearly_full_sectors(S, n_so, n_e):
    """One electron or one hole per spin: no same-spin doubles on one side, so the row sweep's
    pair tables are empty there; both sweeps and the energy against the oracle."""
    w = I.small_case(n_so, n_e, 12, 150 + n_so + n_e)
    ko, ao = O.apply_ansatz(n_so, n_e, w.ops, w.theta, 0)
    go = O.pool_gradients(n_so, w.h, w.g, ko, ao)
    eo = O.energy(n_so, w.h, w.g, ko, ao)[0]
    for sweep in (2, 1):
        c = ctx_for(S, w)
        c.set_option("sweep", sweep)
        c.apply_ansatz(w.ops, w.theta, 0)
        k, a = c.get_state()
        assert_state_equal(k, a, ko, ao)
        assert abs(c.energy()[0] - eo) < TOL
        assert np.abs(c.pool_gradients() - go).max() < TOL
