"""Screening network on the tensor cores against the CPU oracle (oracle/mlp.py).

Each stage is compared with the oracle evaluated on the GPU's own BF16 inputs
to that stage, so a BF16 rounding decision taken differently upstream cannot
propagate: stored activations within one BF16 ulp, FP32 outputs within the
FP32 accumulation bound, gradients within 1e-3 of their scale."""
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


def within_ulp(gpu, ref, a, w):
    """One BF16 ulp of the reference, plus the FP32 accumulation bound of
    each entry (a ReLU input within that bound of zero may land either side)."""
    acc = 2.0 ** -20 * (np.abs(a) @ np.abs(w).T) + 1e-7
    return np.all(np.abs(gpu - ref) <= 2.0 ** -7 * np.abs(ref) + acc)


@pytest.mark.parametrize("n", [128, 300, 1000])
def test_forward_stages(S, n):
    import torch
    rng = np.random.default_rng(n)
    net = S.Mlp(32, 256)
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


@pytest.mark.parametrize("n", [256, 777])
def test_gradients_match_oracle(S, n):
    import torch
    rng = np.random.default_rng(7 + n)
    net = S.Mlp(32, 256)
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
    for name, rname in (("W1", "dW1"), ("b1", "db1"), ("W2", "dW2"), ("b2", "db2"), ("w3", "dw3"), ("b3", "db3")):
        a, b = np.asarray(g[name]), np.asarray(ref[rname])
        scale = max(np.abs(b).max(), 1e-12)
        assert np.abs(a - b).max() <= 1e-3 * scale, (name, np.abs(a - b).max(), scale)
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
    ref = M.forward(x, M.bf16_round(P["W1"]), P["b1"], M.bf16_round(P["W2"]), P["b2"], M.bf16_round(P["w3"]),
                    P["b3"])["y"]
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-2 * max(1.0, np.abs(ref).max())
