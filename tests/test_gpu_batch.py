"""Batched launch: every instance's energy and pool gradient equal the oracle
(small instances) or the single-context path (the full 64-instance workload),
for the persistent kernel under several tilings, for the graph of
per-instance branches, and for the back-to-back comparator; the tuning cache."""
import json

import numpy as np
import pytest

import oracle as O
from paper_2411_07920_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-10

SMALL = [(12, 4, 10, 201, 0), (16, 6, 25, 202, 120), (20, 6, 40, 203, 400), (14, 4, 20, 204, 50),
         (18, 8, 30, 205, 300), (24, 8, 35, 206, 600), (16, 2, 8, 207, 0)]


@pytest.fixture(scope="module")
def S():
    from paper_2411_07920_gb300 import swcs
    return swcs


@pytest.fixture(scope="module")
def small_ref():
    ws = [I.small_case(n_so, n_e, n_ops, seed, n_keep=nk) for (n_so, n_e, n_ops, seed, nk) in SMALL]
    ref = []
    for w in ws:
        ko, ao = O.apply_ansatz(w.n_so, w.n_e, w.ops, w.theta, w.n_keep)
        eo, n2o = O.energy(w.n_so, w.h, w.g, ko, ao)
        ref.append((eo, n2o, O.pool_gradients(w.n_so, w.h, w.g, ko, ao)))
    return ws, ref


def _check_small(b, ws, ref):
    for i in range(len(ws)):
        e, n2, g = b.results(i)
        eo, n2o, go = ref[i]
        assert abs(e - eo) < TOL and abs(n2 - n2o) < 1e-13, (i, e, eo)
        assert np.abs(g - go).max() < TOL, i


@pytest.mark.parametrize("mode,tile,ctas,factor", [
    (0, 4096, 2, 2), (0, 256, 2, 2), (0, 512, 1, 4), (0, 16384, 2, 8), (1, 4096, 2, 2)])
def test_batch_matches_oracle(S, small_ref, mode, tile, ctas, factor):
    ws, ref = small_ref
    b = S.Batch()
    for w in ws:
        b.add(w.h, w.g, w.n_so, w.n_e, w.ops, w.theta, w.n_keep)
    b.set_tuning(mode, tile, ctas, factor)
    b.build(autotune=False)
    for rep in range(2):  # the launch is repeatable: its scheduler words are reset inside the graph
        b.run()
        _check_small(b, ws, ref)
    t = b.tuning()
    assert t["instances"] == len(ws) and t["mode"] == mode
    if mode == 0:
        assert (t["tile"], t["ctas_per_sm"], t["hash_factor"]) == (tile, ctas, factor)
    b.close()


def test_batch_autotune_cache_and_serial_comparator(S, small_ref, tmp_path):
    ws, ref = small_ref
    path = str(tmp_path / "tuning.json")
    tunings = []
    for attempt in range(2):
        b = S.Batch()
        for w in ws:
            b.add(w.h, w.g, w.n_so, w.n_e, w.ops, w.theta, w.n_keep)
        b.build(autotune=True, cache_path=path)
        assert b.from_cache == (attempt == 1)
        b.run()
        _check_small(b, ws, ref)
        t = b.tuning()
        tunings.append((t["mode"], t["tile"], t["ctas_per_sm"], t["hash_factor"]))
        b.run_serial()  # the library's per-instance kernels back to back on one stream
        _check_small(b, ws, ref)
        b.close()
    assert tunings[0] == tunings[1]
    cache = json.load(open(path))
    assert len(cache) == 1 and set(next(iter(cache.values()))) >= {"tile", "ctas_per_sm", "hash_factor"}


def test_batch_64_uneven_instances_match_single_contexts(S):
    """The whole batched workload (64 instances: 16-40 spin-orbitals, 4-12
    electrons, 20-150 gates, N_keep 1e3-1e5) against one context per instance."""
    specs = I.batch_specs(64, 100)
    ws = [I.batch_instance(s) for s in specs]
    b = S.Batch()
    for w in ws:
        b.add(w.h, w.g, w.n_so, w.n_e, w.ops, w.theta, w.n_keep)
    b.build(autotune=False)
    b.run()
    c = S.Context()
    for i, w in enumerate(ws):
        e, n2, g = b.results(i)
        c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
        c.apply_ansatz(w.ops, w.theta, w.n_keep)
        g1 = c.pool_gradients()
        e1, n21 = c.sweep_energy()
        assert abs(e - e1) < TOL and abs(n2 - n21) < 1e-12 * max(1.0, n21), i
        assert np.abs(g - g1).max() < TOL, i
    c.close()
    b.close()
