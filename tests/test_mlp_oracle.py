"""Pins of the screening network's CPU oracle (oracle/mlp.py)."""
import numpy as np

from oracle import mlp as M


def _bf16_reference(f):
    """Nearest BF16 by brute force: the two BF16 neighbours of f, the closer
    one, ties to the even mantissa."""
    f = np.float32(f)
    u = np.array([f], np.float32).view(np.uint32)[0]
    lo = np.uint32(u & 0xFFFF0000)
    hi = np.uint32(lo + 0x10000)
    vlo = np.array([lo], np.uint32).view(np.float32)[0].astype(np.float64)
    vhi = np.array([hi], np.uint32).view(np.float32)[0].astype(np.float64)
    x = float(f)
    dlo, dhi = abs(x - vlo), abs(vhi - x)
    if dlo < dhi or (dlo == dhi and ((lo >> 16) & 1) == 0):
        return vlo
    return vhi


def test_bf16_rounding_matches_brute_force():
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.normal(size=2000).astype(np.float32),
                           np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 3.14159, 0.0, 1e-30,
                                     -7.75e5], np.float32)])
    got = M.bf16_round(vals)
    ref = np.array([_bf16_reference(v) for v in vals])
    assert np.array_equal(got, ref)
    assert M.bf16_round(np.float32(1 + 2 ** -8))[()] == 1.0          # tie to even (down)
    assert M.bf16_round(np.float32(1 + 3 * 2 ** -8))[()] == 1 + 2 ** -6  # tie to even (up)
    assert np.array_equal(M.from_bf16_bits(M.bf16_bits(vals)), got)


def _net(rng, d_in=8, w=16):
    return dict(W1=rng.normal(size=(w, d_in)) * 0.5, b1=rng.normal(size=w) * 0.1,
                W2=rng.normal(size=(w, w)) * 0.3, b2=rng.normal(size=w) * 0.1,
                w3=rng.normal(size=w) * 0.3, b3=0.2)


def test_backward_matches_finite_differences_without_rounding():
    rng = np.random.default_rng(1)
    p = _net(rng)
    x = rng.normal(size=(13, 8))
    t = rng.normal(size=13)
    ident = lambda a: np.asarray(a, np.float64)

    def L(q):
        fw = M.forward(x, q["W1"], q["b1"], q["W2"], q["b2"], q["w3"], q["b3"], rnd=ident)
        return M.loss(fw["y"], t)

    fw = M.forward(x, p["W1"], p["b1"], p["W2"], p["b2"], p["w3"], p["b3"], rnd=ident)
    g = M.backward(x, t, p["W1"], p["W2"], p["w3"], fw, bf16_grads=False, rnd=ident)
    h = 1e-6
    for name, gname in (("W1", "dW1"), ("b1", "db1"), ("W2", "dW2"), ("b2", "db2"), ("w3", "dw3")):
        arr = p[name]
        for idx in [(0,), (3,), (5,)] if arr.ndim == 1 else [(0, 0), (2, 5), (7, 3)]:
            q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
            q[name][idx] += h
            lp = L(q)
            q[name][idx] -= 2 * h
            lm = L(q)
            assert abs((lp - lm) / (2 * h) - g[gname][idx]) < 1e-6
    q = dict(p)
    q["b3"] = p["b3"] + h
    lp = L(q)
    q["b3"] = p["b3"] - h
    assert abs((lp - L(q)) / (2 * h) - g["db3"]) < 1e-6


def test_single_layer_closed_form():
    # with W2 = I, b2 = 0, w3 = 1 and nonnegative first layer, y = sum(relu(x W1^T + b1))
    rng = np.random.default_rng(2)
    x = np.abs(rng.normal(size=(5, 4)))
    W1 = np.abs(rng.normal(size=(6, 4)))
    b1 = np.abs(rng.normal(size=6))
    ident = lambda a: np.asarray(a, np.float64)
    fw = M.forward(x, W1, b1, np.eye(6), np.zeros(6), np.ones(6), 0.0, rnd=ident)
    assert np.allclose(fw["y"], (x @ W1.T + b1).sum(axis=1), rtol=1e-14)
