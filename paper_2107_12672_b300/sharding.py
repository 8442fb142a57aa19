"""Sharding views across ranks (one process per GPU).

Rays, and therefore views, are independent (Alg. 1 runs "in parallel over
all pixels"): each rank renders and differentiates its share of the views
with the volume and TF replicated, and the only exchange is the sum of the
parameter gradients (volume, TF; each camera gradient lives on the rank that
owns the view). Views are assigned greedily by pixel count, largest first,
to the least-loaded rank, so uneven resolutions balance.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_views(views, world: int) -> list:
    """Assignment of view indices to `world` ranks, balanced by pixels."""
    load = [0] * world
    owner = [[] for _ in range(world)]
    order = sorted(range(len(views)), key=lambda i: -(views[i].width * views[i].height))
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[r].append(i)
        load[r] += views[i].width * views[i].height
    return [sorted(o) for o in owner]


def allreduce_gradients(grads: dict, group=None) -> dict:
    """Sum the gradient tensors of every rank in place (volume list, TF,
    and the [n_views][3] camera gradients, zero on views a rank does not
    own). Returns `grads`."""
    for key in ("volume", "tf", "eye", "step"):
        g = grads.get(key)
        if g is None:
            continue
        for t in (g if isinstance(g, list) else [g]):
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return grads


def scatter_camera_gradient(local_eye_grad: torch.Tensor, owned, n_views: int) -> torch.Tensor:
    """Place the camera gradients of a rank's own views into the full
    [n_views][3] array (zeros elsewhere) before the all-reduce."""
    full = torch.zeros((n_views, 3), dtype=local_eye_grad.dtype, device=local_eye_grad.device)
    full[list(owned)] = local_eye_grad
    return full
