"""Learned pool screening around the C ABI (orchestration only).

The pool gradient of ADAPT step 4 (Sec. II.C) is evaluated exactly for the
operators a small network ranks highest.  Everything numerical runs in the
library: features (swcs_pool_features_dev), exact gradients
(swcs_pool_gradients_dev), targets (swcs_log_abs_dev), the network's forward,
backward and Adam steps (swcs_mlp_*), top-k selection and the subset sweep
(swcs_pool_screen_dev, swcs_pool_gradients_dev with a subset).  This module
only moves device tensors between those calls and draws minibatch indices.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import inputs as I
from . import swcs


def init_params(width: int = 256, d_in: int = 32, seed: int = 0) -> np.ndarray:
    """He-initialised parameters in the library's order."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(size=width * d_in) * np.sqrt(2.0 / d_in), np.zeros(width),
             rng.normal(size=width * width) * np.sqrt(2.0 / width), np.zeros(width),
             rng.normal(size=width) * np.sqrt(1.0 / width), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def state_samples(ctx: swcs.Context):
    """(features [pool, 32] BF16 bits, targets max(log10|g|, -10) [pool]) of the current state."""
    P = ctx.pool_size()
    x = torch.empty((P, 32), dtype=torch.int16, device="cuda")
    ctx.pool_features_dev(x)
    g = torch.empty(P, dtype=torch.float64, device="cuda")
    ctx.pool_gradients_dev(g)
    t = torch.empty(P, dtype=torch.float32, device="cuda")
    swcs.log_abs_dev(g, t)
    return x, t, g


def training_set(specs, seed: int = 0):
    """Exact pool gradients generated by the method itself on small systems.

    specs: list of (n_so, n_e, n_ops, seed, n_keep); several prefixes of each
    ansatz give several states per system."""
    xs, ts = [], []
    for (n_so, n_e, n_ops, sd, n_keep) in specs:
        w = I.small_case(n_so, n_e, n_ops, sd, n_keep=n_keep)
        with swcs.Context() as c:
            c.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
            for m in sorted({max(1, len(w.ops) // 3), max(1, 2 * len(w.ops) // 3), len(w.ops)}):
                c.apply_ansatz(w.ops[:m], w.theta[:m], n_keep)
                x, t, _ = state_samples(c)
                xs.append(x)
                ts.append(t)
    return torch.cat(xs), torch.cat(ts)


def default_specs():
    """States from the two small workload families (12 spin-orbitals / 4
    electrons without truncation; 28 / 8 truncated), several seeds each."""
    specs = [(12, 4, 10, s, 0) for s in (1, 11, 21, 31)]
    specs += [(28, 8, 60, s, 20000) for s in (2, 12, 22)]
    specs += [(20, 6, 40, s, 2000) for s in (5, 15)]
    return specs


def train(net: swcs.Mlp, X, T, steps: int = 800, batch: int = 8192, lr: float = 3e-3, seed: int = 0):
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    hist = []
    for it in range(steps):
        idx = torch.from_numpy(rng.integers(0, n, size=min(batch, n))).cuda()
        xb = X.index_select(0, idx).contiguous()
        tb = T.index_select(0, idx).contiguous()
        net.train_step_dev(xb, tb, lr * (0.5 if it > steps * 0.7 else 1.0), loss)
        if it % 100 == 0 or it == steps - 1:
            net.sync()
            hist.append((it, loss.item()))
    return hist


def evaluate(ctx: swcs.Context, net: swcs.Mlp, frac: float = 0.05, full=None):
    """Screened vs full pool sweep on the context's current state.

    Returns recall of the exact argmax and of the exact top-10, the ranks, and
    the wall times of the two sweeps (both synchronised)."""
    P = ctx.pool_size()
    if full is None:
        g_full = torch.empty(P, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.pool_gradients_dev(g_full)
        torch.cuda.synchronize()
        t_full = time.perf_counter() - t0
    else:
        g_full, t_full = full
    sub = torch.empty(P, dtype=torch.int64, device="cuda")
    g_sub = torch.empty(P, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k = ctx.pool_screen_dev(net, frac, sub)
    ctx.pool_gradients_dev(g_sub, sub[:k])
    torch.cuda.synchronize()
    t_scr = time.perf_counter() - t0
    gf = g_full.cpu().numpy()
    chosen = sub[:k].cpu().numpy()
    gs = g_sub.cpu().numpy()[chosen]
    top = np.argsort(-np.abs(gf))
    sel = set(chosen.tolist())
    argmax_exact = int(top[0])
    argmax_screened = int(chosen[np.argmax(np.abs(gs))])
    return dict(recall_argmax=float(argmax_exact in sel), recall_top10=float(np.mean([t in sel for t in top[:10]])),
                same_argmax=argmax_exact == argmax_screened, subset=int(k), pool=int(P),
                max_abs_err_on_subset=float(np.abs(gs - gf[chosen]).max()), t_full=t_full, t_screened=t_scr,
                speedup=t_full / t_scr if t_scr > 0 else None)
