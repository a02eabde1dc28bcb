"""Launch-shape autotuner for akmc_step_n.

Times candidate shapes (warps per voxel-CTA, CTAs per SM) on a scratch batch
built from the same descriptors (the caller's batch is never stepped), picks
the fastest and caches the choice per workload key for the process.
"""
from __future__ import annotations

import collections

import numpy as np

from .akmc import Batch

_cache = {}


def workload_key(descs):
    """Key: model/precision mix, edge lengths and vacancy counts (bucketed)."""
    c = collections.Counter((d.model, d.precision, d.L, min(d.n_vac, 8)) for d in descs)
    return tuple(sorted(c.items()))


def tune(descs, model, events=2000, candidates=((8, 0), (16, 0), (4, 0), (2, 0), (8, 1), (4, 2)), sample=1024):
    """Return (warps, ctas_per_sm) with the highest events/s on a scratch copy
    of up to `sample` of the voxels."""
    import torch
    key = workload_key(descs)
    if key in _cache:
        return _cache[key]
    descs = list(descs)[:sample]
    scratch = Batch(descs, model)
    best, best_rate = candidates[0], -1.0
    n_ev = np.full(len(descs), events, np.uint64)
    for warps, per_sm in candidates:
        scratch.set_launch(warps, per_sm)
        scratch.step(n_ev // 4)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s.record()
        scratch.step(n_ev)
        e.record()
        torch.cuda.synchronize()
        rate = float(n_ev.sum()) / (s.elapsed_time(e) * 1e-3)
        if rate > best_rate:
            best, best_rate = (warps, per_sm), rate
    scratch.close()
    del scratch
    _cache[key] = best
    return best
