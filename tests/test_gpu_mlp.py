"""Screening network on the tensor cores against the CPU oracle (oracle/mlp.py).

Each stage is compared with the oracle evaluated on the GPU's own BF16 inputs
to that stage, so a BF16 rounding decision taken differently upstream cannot
propagate: stored activations within one BF16 ulp, FP32 outputs within the
FP32 accumulation bound.  Gradients and the end-to-end forward are held to
bounds derived from the arithmetic (bound_* below): every FP32 accumulation
of K terms errs by at most K * 2^-23 times the sum of the terms' magnitudes
(any order, rounding or truncation), and a BF16-rounded intermediate can
differ from the oracle's by one BF16 step only where its value lies within
its propagated error of a rounding boundary."""
import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu


def he_params(rng, d_in, w):
    p = np.zeros(w * d_in + w + w * w + w + w + 1, np.float32)
    o = 0
    p[o:o + w * d_in] = rng.normal(size=w * d_in) * np.sqrt(2.0 / d_in); o += w * d_in
    p[o:o + w] = rng.normal(size=w) * 0.05; o += w
    p[o:o + w * w] = rng.normal(size=w * w) * np.sqrt(2.0 / w); o += w * w
    p[o:o + w] = rng.normal(size=w) * 0.05; o += w
    p[o:o + w] = rng.normal(size=w) * np.sqrt(1.0 / w); o += w
    p[o] = 0.1
    return p


def unpack(net, flat):
    out = {}
    for k, (o, shape) in net.layout().items():
        n = int(np.prod(shape)) if shape else 1
        out[k] = flat[o:o + n].astype(np.float64).reshape(shape) if shape else float(flat[o])
    return out


@pytest.fixture(scope="module")
def S():
    from paper_2411_07920_gb300 import swcs
    return swcs


U32 = 2.0 ** -24      # FP32 unit roundoff (one rounded operation)
U_ACC = 2.0 ** -23    # per term of an FP32 accumulation, any order and rounding mode


def gamma(k):
    return k * U_ACC


def bf16_step(v, r):
    """Bound on |bf16(v') - bf16(v)| over |v' - v| <= r: 0 where no BF16
    rounding boundary lies within r of v, else r plus one BF16 spacing."""
    a = np.abs(v) + r
    ulp = np.where(a > 0, 2.0 ** (np.floor(np.log2(np.where(a > 0, a, 1.0))) - 7), 0.0)
    risky = M.bf16_round(v - r) != M.bf16_round(v + r)
    return np.where(risky, r + ulp, 0.0)


def bound_grads(x, t, W1, W2, w3, fw):
    """Per-entry bounds of |GPU - oracle| for every gradient, following the
    GPU's order of work: dy = 2 (y - t) / B and dZ2 = bf16(dy w3 [H2 > 0]) in
    FP32 (a few roundings), dH1 = dZ2 W2 and the weight gradients as FP32
    accumulations over 256 (width) or B (batch) terms, dZ1 = bf16(dH1 [H1 > 0])."""
    B, W = fw["H1"].shape
    y = fw["y"]
    dy = 2.0 * (y - np.asarray(t, np.float64)) / B
    ady = np.abs(dy)
    v2 = np.outer(dy, w3) * (fw["H2"] > 0)
    D2 = bf16_step(v2, 4 * U32 * np.abs(v2))
    dZ2 = M.bf16_round(v2)
    H1a, H2a, xa = np.abs(fw["H1"]), np.abs(fw["H2"]), np.abs(x)
    out = {}
    out["dw3"] = (gamma(B) + 3 * U32) * (H2a.T @ ady)
    out["db3"] = (gamma(B) + 3 * U32) * ady.sum()
    out["db2"] = D2.sum(axis=0) + gamma(B) * np.abs(dZ2).sum(axis=0)
    out["dW2"] = D2.T @ H1a + gamma(B) * (np.abs(dZ2).T @ H1a)
    r1 = (D2 @ np.abs(W2) + gamma(W) * (np.abs(dZ2) @ np.abs(W2))) * (fw["H1"] > 0)
    v1 = (dZ2 @ W2) * (fw["H1"] > 0)
    D1 = bf16_step(v1, r1)
    dZ1 = M.bf16_round(v1)
    out["db1"] = D1.sum(axis=0) + gamma(B) * np.abs(dZ1).sum(axis=0)
    out["dW1"] = D1.T @ xa + gamma(B) * (np.abs(dZ1).T @ xa)
    return out


def bound_forward(x, W1, b1, W2, b2, w3):
    """Bound of |y_GPU - y_oracle| when both start from x: FP32 accumulations
    of the three contractions, one BF16 step for each stored activation that
    lies within its propagated error of a rounding boundary."""
    d_in, W = W1.shape[1], W1.shape[0]
    fw = M.forward(x, W1, b1, W2, b2, w3, 0.0)
    Z1 = M.linear(x, W1, b1)
    r1 = gamma(d_in + 1) * (np.abs(x) @ np.abs(W1).T + np.abs(b1))
    D1 = bf16_step(np.maximum(Z1, 0.0), r1)
    H1a = np.abs(fw["H1"]) + D1
    Z2 = M.linear(fw["H1"], W2, b2)
    r2 = D1 @ np.abs(W2).T + gamma(W + 1) * (H1a @ np.abs(W2).T + np.abs(b2))
    D2 = bf16_step(np.maximum(Z2, 0.0), r2)
    H2a = np.abs(fw["H2"]) + D2
    return D2 @ np.abs(w3) + gamma(W + 1) * (H2a @ np.abs(w3) + 1.0)


def within_ulp(gpu, ref, a, w):
    """One BF16 ulp of the reference, plus the FP32 accumulation bound of
    each entry (a ReLU input within that bound of zero may land either side)."""
    acc = 2.0 ** -20 * (np.abs(a) @ np.abs(w).T) + 1e-7
    return np.all(np.abs(gpu - ref) <= 2.0 ** -7 * np.abs(ref) + acc)


@pytest.mark.parametrize("pipeline", [1, 0])
@pytest.mark.parametrize("n", [128, 300, 1000])
def test_forward_stages(S, n, pipeline):
    import torch
    rng = np.random.default_rng(n)
    net = S.Mlp(32, 256)
    net.set_option("gemm_pipeline", pipeline)
    flat = he_params(rng, 32, 256)
    net.set_params(flat)
    P = unpack(net, flat)
    W1, W2, w3 = M.bf16_round(P["W1"]), M.bf16_round(P["W2"]), M.bf16_round(P["w3"])
    x = M.bf16_round(rng.normal(size=(n, 32)))
    d_x = torch.from_numpy(M.bf16_bits(x).view(np.int16).copy()).cuda()
    d_t = torch.zeros(n, dtype=torch.float32, device="cuda")
    d_loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.grad_dev(d_x, d_t, None, d_loss)
    H1b, H2b, y = net.activations(n)
    H1 = M.from_bf16_bits(H1b)
    H2 = M.from_bf16_bits(H2b)
    ref1 = M.bf16_round(np.maximum(M.linear(x, W1, P["b1"]), 0))
    assert within_ulp(H1, ref1, x, W1)
    ref2 = M.bf16_round(np.maximum(M.linear(H1, W2, P["b2"]), 0))
    assert within_ulp(H2, ref2, H1, W2)
    yref = H2 @ w3 + P["b3"]
    assert np.abs(y - yref).max() <= 1e-5 * (np.abs(H2) @ np.abs(w3)).max() + 1e-6
    # the inference entry point gives the same y
    d_y = torch.zeros(n, dtype=torch.float32, device="cuda")
    net.forward_dev(d_x, d_y)
    torch.cuda.synchronize()
    assert np.array_equal(d_y.cpu().numpy(), y)
    net.close()


@pytest.mark.parametrize("pipeline", [1, 0])
@pytest.mark.parametrize("n", [256, 777, 5000])
def test_gradients_match_oracle(S, n, pipeline):
    """Both GEMM paths (TMA-pipelined with K split over CTAs for the weight gradients; staged with plain
    loads) within the bounds derived for any FP32 summation order."""
    import torch
    rng = np.random.default_rng(7 + n)
    net = S.Mlp(32, 256)
    net.set_option("gemm_pipeline", pipeline)
    flat = he_params(rng, 32, 256)
    net.set_params(flat)
    P = unpack(net, flat)
    W1, W2, w3 = M.bf16_round(P["W1"]), M.bf16_round(P["W2"]), M.bf16_round(P["w3"])
    x = M.bf16_round(rng.normal(size=(n, 32)))
    t = rng.normal(size=n).astype(np.float32)
    d_x = torch.from_numpy(M.bf16_bits(x).view(np.int16).copy()).cuda()
    d_t = torch.from_numpy(t).cuda()
    d_g = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
    d_loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.grad_dev(d_x, d_t, d_g, d_loss)
    H1b, H2b, y = net.activations(n)
    fw = dict(H1=M.from_bf16_bits(H1b), H2=M.from_bf16_bits(H2b), y=y.astype(np.float64))
    ref = M.backward(x, t, W1, W2, w3, fw)
    g = unpack(net, d_g.cpu().numpy())
    assert abs(d_loss.item() - M.loss(y, t)) < 1e-5 * max(1.0, M.loss(y, t))
    bound = bound_grads(x, t, W1, W2, w3, fw)
    for name, rname in (("W1", "dW1"), ("b1", "db1"), ("W2", "dW2"), ("b2", "db2"), ("w3", "dw3"), ("b3", "db3")):
        a, b = np.asarray(g[name]), np.asarray(ref[rname])
        # the derived bound, plus FP32 storage of the result itself
        tol = np.asarray(bound[rname]) + 2 * U32 * np.abs(b) + 1e-30
        assert np.all(np.abs(a - b) <= tol), (name, np.abs(a - b).max(), float(np.max(tol)))
        # and the bound is a real constraint: far below the gradient's own scale
        assert float(np.max(tol)) < 1e-2 * max(np.abs(b).max(), 1e-12), name
    net.close()


def test_training_reduces_loss(S):
    import torch
    rng = np.random.default_rng(3)
    net = S.Mlp(32, 256)
    net.set_params(he_params(rng, 32, 256))
    n = 4096
    x = M.bf16_round(rng.normal(size=(n, 32)))
    t = (np.sin(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2]).astype(np.float32)
    d_x = torch.from_numpy(M.bf16_bits(x).view(np.int16).copy()).cuda()
    d_t = torch.from_numpy(t).cuda()
    d_loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    losses = []
    for it in range(300):
        net.train_step_dev(d_x, d_t, 3e-3, d_loss)
        if it in (0, 299):
            net.sync()
            losses.append(d_loss.item())
    assert losses[1] < 0.2 * losses[0]
    net.close()


@pytest.mark.parametrize("n,d_in,width", [(5, 32, 256), (1000, 32, 256), (128 * 152 * 3 + 77, 32, 256),
                                          (4099, 64, 128), (777, 32, 64), (300, 64, 256),
                                          (301600, 32, 256)])
def test_fused_forward_is_bit_identical(S, n, d_in, width):
    """The fused inference kernel (TMA, both layers on chip) returns exactly the
    layer-by-layer result, for partial tiles, several tiles per CTA and other
    shapes (64 x 256 exceeds its shared memory and runs layer by layer)."""
    import torch
    rng = np.random.default_rng(n + d_in)
    net = S.Mlp(d_in, width)
    flat = he_params(rng, d_in, width)
    net.set_params(flat)
    x = M.bf16_round(rng.normal(size=(n, d_in)))
    d_x = torch.from_numpy(M.bf16_bits(x).view(np.int16).copy()).cuda()
    y_ref = torch.empty(n, dtype=torch.float32, device="cuda")
    y = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    net.forward_dev(d_x, y_ref)
    net.predict_dev(d_x, y)
    net.sync()
    assert torch.equal(y, y_ref)
    P = unpack(net, flat)
    W1, W2, w3 = M.bf16_round(P["W1"]), M.bf16_round(P["W2"]), M.bf16_round(P["w3"])
    ref = M.forward(x, W1, P["b1"], W2, P["b2"], w3, P["b3"])["y"]
    tol = bound_forward(x, W1, P["b1"], W2, P["b2"], w3) + 2 * U32 * np.abs(ref)
    assert np.all(np.abs(y.cpu().numpy() - ref) <= tol), np.abs(y.cpu().numpy() - ref).max()


@pytest.mark.parametrize("n,d_in,width", [(4096, 32, 256), (1000, 64, 128), (333, 32, 64)])
def test_gemm_paths_agree(S, n, d_in, width):
    """The forward activations of the two GEMM paths are bit for bit the same (the tensor cores see the same
    sequence of K = 16 steps); the gradients agree within the bound of two FP32 summation orders."""
    import torch
    rng = np.random.default_rng(n + d_in)
    flat = he_params(rng, d_in, width)
    x = M.bf16_round(rng.normal(size=(n, d_in)))
    t = rng.normal(size=n).astype(np.float32)
    d_x = torch.from_numpy(M.bf16_bits(x).view(np.int16).copy()).cuda()
    d_t = torch.from_numpy(t).cuda()
    out = []
    for pipeline in (1, 0):
        net = S.Mlp(d_in, width)
        net.set_option("gemm_pipeline", pipeline)
        net.set_params(flat)
        d_g = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
        d_loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        net.grad_dev(d_x, d_t, d_g, d_loss)
        H1b, H2b, y = net.activations(n)
        out.append((H1b, H2b, y, d_g.cpu().numpy().astype(np.float64), unpack(net, flat)))
        net.close()
    (H1a, H2a, ya, ga, P), (H1s, H2s, ys, gs, _) = out
    assert np.array_equal(H1a, H1s) and np.array_equal(H2a, H2s) and np.array_equal(ya, ys)
    # every gradient is a sum over the n rows of the batch in an order that atomics or the K split decide:
    # dW2 = dZ2^T H1 and dW1 = dZ1^T X on the tensor cores, dw3, db3, db2, db1 by FP32 atomics.  Two orders
    # of the same terms differ by at most 2 gamma(n + 2) sum |terms| (the + 2 covers the FP32 products with dy;
    # |dZ| is bounded from above, the BF16 rounding of dZ2 and dZ1 adding at most 2^-8 each)
    H1, H2 = M.from_bf16_bits(H1a), M.from_bf16_bits(H2a)
    W2, w3 = M.bf16_round(P["W2"]), M.bf16_round(P["w3"])
    dy = np.abs(2.0 * (ya.astype(np.float64) - t) / n) * (1 + 2.0 ** -20)
    adZ2 = np.outer(dy, np.abs(w3)) * (H2 > 0) * (1 + 2.0 ** -7)
    adZ1 = (adZ2 @ np.abs(W2)) * (H1 > 0) * (1 + 2.0 ** -7)
    G = 2 * gamma(n + 2)
    bound = {"W2": G * (adZ2.T @ np.abs(H1)), "W1": G * (adZ1.T @ np.abs(x)), "w3": G * (dy @ np.abs(H2)),
             "b3": G * dy.sum(), "b2": G * adZ2.sum(axis=0), "b1": G * adZ1.sum(axis=0)}
    A, Sg = unpack_grad(P, ga), unpack_grad(P, gs)
    for name in A:
        assert np.all(np.abs(A[name] - Sg[name]) <= bound[name] + 1e-30), (name, np.abs(A[name] - Sg[name]).max())


def unpack_grad(P, g):
    """The gradient vector cut like the parameter dictionary P."""
    out, o = {}, 0
    for name in ("W1", "b1", "W2", "b2", "w3", "b3"):
        k = int(np.asarray(P[name]).size)
        out[name] = g[o:o + k].reshape(np.asarray(P[name]).shape)
        o += k
    return out


def test_mlp_option_errors(S):
    net = S.Mlp(32, 256)
    with pytest.raises(Exception):
        net.set_option("gemm_pipeline", 2)
    with pytest.raises(Exception):
        net.set_option("no_such_option", 1)
    net.close()
