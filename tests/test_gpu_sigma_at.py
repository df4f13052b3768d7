"""sigma_E = (H psi)_E at arbitrary determinants of the sector, read out of
the pool sweep's alpha-string rows (swcs_sigma_at), against the oracle's pull
form (each E from its own connections): external determinants one excitation
away, two away, disconnected ones (sigma = 0), members of the state, repeats,
several launch shapes; and the argument checks."""
import numpy as np
import pytest

import oracle as O
from paper_2411_07920_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _random_dets(n_so, n_e, count, rng):
    m, ks = n_so // 2, n_e // 2
    out = []
    for _ in range(count):
        al = rng.choice(m, ks, replace=False)
        be = rng.choice(m, ks, replace=False)
        d = 0
        for p in al:
            d |= 1 << (2 * int(p))
        for p in be:
            d |= 1 << (2 * int(p) + 1)
        out.append(d)
    return out


def _neighbours(k, n_so, count, rng, n_exc):
    out = []
    for _ in range(count):
        d = int(k[rng.integers(len(k))])
        for _ in range(n_exc):
            spin = int(rng.integers(2))
            occ = [p for p in range(spin, n_so, 2) if (d >> p) & 1]
            vir = [p for p in range(spin, n_so, 2) if not (d >> p) & 1]
            d ^= (1 << int(rng.choice(occ))) | (1 << int(rng.choice(vir)))
        out.append(d)
    return out


@pytest.mark.parametrize("n_so,n_e,n_ops,seed,n_keep,cluster", [
    (12, 4, 10, 1, 0, 2), (20, 6, 40, 81, 500, 1), (20, 6, 40, 81, 500, 4), (28, 8, 60, 2, 3000, 2),
    (64, 6, 8, 83, 300, 2)])
def test_sigma_at_matches_oracle(n_so, n_e, n_ops, seed, n_keep, cluster):
    from paper_2411_07920_gb300 import swcs
    w = I.small_case(n_so, n_e, n_ops, seed, n_keep=n_keep)
    rng = np.random.default_rng(seed)
    with swcs.Context() as c:
        c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
        c.set_option("cluster", cluster)
        c.apply_ansatz(w.ops, w.theta, n_keep)
        k, a = c.get_state()
        at = (_neighbours(k, n_so, 60, rng, 1) + _neighbours(k, n_so, 60, rng, 2) + _random_dets(n_so, n_e, 30, rng)
              + [int(x) for x in k[rng.choice(len(k), min(len(k), 20), replace=False)]])
        at = np.array(at + at[:5], np.uint64)  # repeats are answered in place
        got = c.sigma_at(at)
        want = O.sigma_at(w.n_so, w.h, w.g, k, a, at)
        assert np.abs(got - want).max() < TOL, np.abs(got - want).max()
        assert np.abs(want).max() > 1e-3
        if n_so >= 28:
            assert (want == 0.0).any()  # some random samples are disconnected from the state
        # the sweep rows are left clean: the pool gradient afterwards is unchanged
        g = c.pool_gradients()
        go = O.pool_gradients(w.n_so, w.h, w.g, k, a)
        assert np.abs(g - go).max() < TOL


def test_sigma_at_rejects_determinants_outside_the_sector():
    from paper_2411_07920_gb300 import swcs
    w = I.small_case(12, 4, 10, 1)
    with swcs.Context() as c:
        c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
        c.apply_ansatz(w.ops, w.theta, 0)
        for bad in (0b11, 0b1111 << 12, 0b0101 | (1 << 13), 0b0101 | (0b0101 << 8)):  # count, bits >= n_so, S_z
            with pytest.raises(swcs.SwcsError):
                c.sigma_at(np.array([bad], np.uint64))
        assert len(c.sigma_at(np.zeros(0, np.uint64))) == 0
