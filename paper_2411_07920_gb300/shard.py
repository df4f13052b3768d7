"""The pool sweep spread over the ranks of a torch.distributed process group.

ADAPT step 4 (Sec. II.C) forms sigma_E = (H psi)_E on every determinant E
connected to the state and contracts it into the pool gradient.  With one
process per GPU, each holding the same state, rank r forms sigma only for the
E whose alpha string has colex rank = r (mod world size) -- whole rows of the
row sweep -- so every sigma_E is formed once.  The partial gradients and
energy numerators are then summed by one all-reduce; <psi|psi> is the same on
every rank and enters once.  The arithmetic runs in the library
(swcs_pool_gradients_partial_dev); this module only moves its two outputs
through the collective.
"""
from __future__ import annotations


def sharded_pool_gradients(ctx, group=None, device=None):
    """(g, E) of ctx's current state, the sweep split over the ranks of
    `group` (default: the world).  ctx: a swcs.Context on this rank's GPU.
    Returns a float64 tensor g[pool_size] on `device` and the energy."""
    import torch
    import torch.distributed as dist

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else torch.device("cpu")
    P = ctx.pool_size()
    buf = torch.empty(P + 2, dtype=torch.float64, device=device)
    ctx.pool_gradients_partial_dev(rank, world, buf[:P], buf[P:])
    if rank != 0:
        buf[P + 1] = 0.0  # <psi|psi> enters the sum once
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    norm2 = buf[P + 1]
    return 2.0 * buf[:P] / norm2, float(buf[P] / norm2)
