"""Voxel sharding across ranks (one process per GPU).

Voxels are independent periodic boxes (no exchange between them), so a
multi-GPU run gives every rank its own voxels and needs no collective on the
data path: rank r takes uids [r*n, (r+1)*n) with per-voxel seeds derived from
the uid.  The only collective is the max-over-ranks of the timed region.
"""
from __future__ import annotations

import dataclasses


def rank_descs(descs, rank: int, seed_fn):
    """The rank's copy of a per-rank workload: uids offset by rank*len(descs),
    seeds recomputed from the new uid with seed_fn(uid)."""
    n = len(descs)
    out = []
    for d in descs:
        uid = int(d.uid) + rank * n
        out.append(dataclasses.replace(d, uid=uid, seed=int(seed_fn(uid))))
    return out


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a float over all ranks of the default process group (or value
    itself without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
