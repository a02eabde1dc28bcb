"""Declared ties (reading R9 of the event order): GPU and oracle rates differ
by ~1e-14 relative (CUDA's exp/log against the host's), so their event
sequences can part only where the uniform t = u1 R falls within that distance
of a boundary between two events' cumulative rates.  These helpers measure
the oracle's margin at an event; a margin below 1e-12 of R is a declared tie,
after which a trajectory test re-seeds instead of failing."""
import numpy as np

import oracle

TIE_MARGIN = 1e-12


def boundary_margin(desc, model, n):
    """Before event n of the oracle's trajectory of `desc`: the distance of
    t = u1 R to the nearest cumulative-rate boundary (event order 8 slot + dir),
    over R, and the event index a linear scan selects."""
    o = oracle.Voxel(desc, model)
    if n:
        o.step(n)
    r = o.state()["rates"].ravel()
    R = o.total_rate()
    u1, _ = oracle.event_uniforms(desc.seed, desc.uid, n)
    t = u1 * R
    c = np.cumsum(r)
    return float(np.min(np.abs(c - t)) / R), int(np.searchsorted(c, t, side="right"))


def is_declared_tie(desc, model, g_log, o_log):
    """False when the two event logs agree; True when they first differ at a
    declared tie; raises AssertionError when they differ anywhere else."""
    bad = np.flatnonzero(np.asarray(g_log) != np.asarray(o_log))
    if bad.size == 0:
        return False
    n = int(bad[0])
    margin, _ = boundary_margin(desc, model, n)
    assert margin < TIE_MARGIN, "event logs differ at event %d, boundary margin %.3g of R (not a tie)" % (n, margin)
    return True
