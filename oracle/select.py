"""TEST INFRASTRUCTURE ONLY: float64 reference of the global masked softmax
selection (logit form of the event selection, Eq. 1-2).

For each segment (one system's concatenated candidate-transition logits):
  z_hat_j = z_j / tau if admissible (mask != 0 and z_j finite), else -inf  (Eq. 1)
  p = softmax(z_hat)                                                       (Eq. 2)
and one index is drawn by inverse CDF: the first j with
sum_{i <= j} exp(z_hat_i - M) > u * sum_i exp(z_hat_i - M), M = max z_hat.
The uniform u of segment s is 53 bits of Philox4x32-10 (the oracle's own
implementation) with key = seed and counter (counter_lo, counter_hi, s,
0x53454c45): u = ((x0 << 21) | (x1 >> 11)) * 2^-53.
Only tests/ and bench.py's baseline leg use this module.
"""
from __future__ import annotations

import numpy as np

from . import philox4x32_10

STREAM = 0x53454C45


def uniform(seed: int, counter: int, s: int) -> float:
    c = [counter & 0xFFFFFFFF, (counter >> 32) & 0xFFFFFFFF, s & 0xFFFFFFFF, STREAM]
    k = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    x = philox4x32_10(c, k)
    m = (x[0] << 21) | (x[1] >> 11)
    return m * 2.0 ** -53


def softmax_probs(z, tau=1.0, mask=None):
    """Probabilities of Eq. 2 over one segment (float64); zeros where masked."""
    z = np.asarray(z, dtype=np.float64)
    ok = np.isfinite(z)
    if mask is not None:
        ok &= np.asarray(mask) != 0
    if not ok.any():
        return np.zeros_like(z), ok
    zh = np.where(ok, z / tau, -np.inf)
    w = np.exp(zh - zh[ok].max())
    return w / w.sum(), ok


def select_one(z, u, tau=1.0, mask=None):
    """(index, log p, margin): the inverse-CDF choice for uniform u, and the
    distance of u*W from the nearest running-sum boundary relative to W."""
    z = np.asarray(z, dtype=np.float64)
    ok = np.isfinite(z)
    if mask is not None:
        ok &= np.asarray(mask) != 0
    if not ok.any():
        return -1, float("nan"), float("inf")
    zh = np.where(ok, z / tau, -np.inf)
    M = zh[ok].max()
    w = np.exp(zh - M)
    c = np.cumsum(w)
    W = c[-1]
    t = u * W
    j = int(np.searchsorted(c, t, side="right"))
    j = min(j, z.size - 1)
    margin = float(np.min(np.abs(c - t)) / W)
    return j, float(zh[j] - M - np.log(W)), margin


def select_segments(logits, offsets, tau=1.0, seed=0, counter=0, mask=None):
    """select_one for every segment with its Philox uniform."""
    logits = np.asarray(logits)
    out = []
    for s in range(len(offsets) - 1):
        b, e = int(offsets[s]), int(offsets[s + 1])
        u = uniform(seed, counter, s)
        out.append(select_one(logits[b:e], u, tau, None if mask is None else mask[b:e]))
    return out
