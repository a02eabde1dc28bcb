"""Pins of the declared-tie helper against the oracle's own selection: the
linear scan of the cumulative rates at t = u1 R picks the event the oracle's
tree descent logged, at a margin far above the tie threshold."""
import numpy as np

import oracle
import synth
from ties import TIE_MARGIN, boundary_margin, is_declared_tie


def test_scan_index_equals_logged_event(model):
    d = synth.VoxelDesc(5, 4, (0.10, 0.08, 0.06), 543.0, synth.PAIR_MODEL, synth.PREC_FP64, seed=2, uid=11)
    log = oracle.Voxel(d, model).step(60, log=True)
    for n in (0, 1, 17, 59):
        margin, k = boundary_margin(d, model, n)
        assert k == log[n]
        assert TIE_MARGIN < margin < 1.0


def test_agreeing_logs_are_no_tie(model):
    d = synth.config_plain_pair()[0]
    log = oracle.Voxel(d, model).step(30, log=True)
    assert is_declared_tie(d, model, log, log) is False
    bad = log.copy()
    bad[7] = (bad[7] + 1) % 8
    try:
        is_declared_tie(d, model, bad, log)
        raise RuntimeError("a divergence far from any boundary must fail")
    except AssertionError as e:
        assert "event 7" in str(e)
