"""CPU oracle of the screening network (test infrastructure only).

The network maps per-operator features x (BF16) to a predicted log|g_k|:
  Z1 = x W1^T + b1,   H1 = bf16(relu(Z1))
  Z2 = H1 W2^T + b2,  H2 = bf16(relu(Z2))
  y  = H2 . w3 + b3
with BF16 weights W1, W2, w3 and FP32 biases; the loss is the mean squared
error against the targets.  Each stage is written out in FP64 from its
definition (plain numpy), taking the BF16-rounded tensors as inputs, so that
the GPU's FP32-accumulated stages can be compared stage by stage.

Parity status: pinned by tests/test_mlp_oracle.py (finite differences of the
loss in FP64, closed-form single-layer cases, bf16 rounding against
numpy's round-half-even on the float32 bit pattern).
"""
from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def bf16_bits(a) -> np.ndarray:
    """BF16 bit patterns (uint16) of bf16_round(a)."""
    f = bf16_round(a).astype(np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


def from_bf16_bits(b) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


def linear(x, w, b=None):
    """x @ w^T (+ b), FP64."""
    z = np.asarray(x, np.float64) @ np.asarray(w, np.float64).T
    return z if b is None else z + np.asarray(b, np.float64)


def forward(x, W1, b1, W2, b2, w3, b3, rnd=bf16_round):
    """rnd: rounding of the stored activations (identity for smooth checks)."""
    Z1 = linear(x, W1, b1)
    H1 = rnd(np.maximum(Z1, 0.0))
    Z2 = linear(H1, W2, b2)
    H2 = rnd(np.maximum(Z2, 0.0))
    y = H2 @ np.asarray(w3, np.float64) + float(b3)
    return dict(Z1=Z1, H1=H1, Z2=Z2, H2=H2, y=y)


def loss(y, t):
    d = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    return float(np.mean(d * d))


def backward(x, t, W1, W2, w3, fw, bf16_grads=True, rnd=bf16_round):
    """Gradients of the mean squared error.  With bf16_grads the two
    pre-activation gradients are rounded to BF16 before the weight-gradient
    contractions, as the tensor-core kernels consume them."""
    B = x.shape[0]
    dy = 2.0 * (fw["y"] - np.asarray(t, np.float64)) / B
    dw3 = fw["H2"].T @ dy
    db3 = float(dy.sum())
    dZ2 = np.outer(dy, np.asarray(w3, np.float64)) * (fw["H2"] > 0)
    if bf16_grads:
        dZ2 = rnd(dZ2)
    dW2 = dZ2.T @ fw["H1"]
    db2 = dZ2.sum(axis=0)
    dH1 = dZ2 @ np.asarray(W2, np.float64)
    dZ1 = dH1 * (fw["H1"] > 0)
    if bf16_grads:
        dZ1 = rnd(dZ1)
    dW1 = dZ1.T @ np.asarray(x, np.float64)
    db1 = dZ1.sum(axis=0)
    return dict(dy=dy, dw3=dw3, db3=db3, dZ2=dZ2, dW2=dW2, db2=db2, dH1=dH1, dZ1=dZ1, dW1=dW1, db1=db1)
