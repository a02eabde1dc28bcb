"""GPU parity of the logit-form global selection (akmc_select_logits, Eq. 1-2)
against the float64 reference oracle/select.py.

The GPU evaluates exp in FP32 and sums the weights exactly in 2^-32 fixed
point; the reference uses float64 throughout.  Selected indices must agree
except where the reference's u*W lies within 4e-6 W of a running-sum
boundary (a declared tie: rounding of the FP32 weights can move the boundary
that far); log-probabilities within 2e-5 absolute.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.select as SEL
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2604_24091_gb300 import AkmcError, Batch, SelectPlan, select_logits  # noqa: E402

TIE = 4e-6


def _compare(logits, offsets, tau, seed, counter, mask=None):
    plan = SelectPlan(offsets)
    lt = torch.from_numpy(logits).cuda()
    mt = torch.from_numpy(mask).cuda() if mask is not None else None
    idx, logp = select_logits(plan, lt, tau, seed, counter, mt)
    idx, logp = idx.cpu().numpy(), logp.cpu().numpy()
    ref = SEL.select_segments(logits.astype(np.float64), offsets, tau, seed, counter, mask)
    ties = 0
    for s, (j, lp, margin) in enumerate(ref):
        if j < 0:
            assert idx[s] == -1 and math.isnan(logp[s]), s
            continue
        if idx[s] != j:
            assert margin < TIE, (s, idx[s], j, margin)
            ties += 1
            continue
        assert abs(logp[s] - lp) <= 2e-5 + 1e-6 * abs(lp), (s, logp[s], lp)
    return ties


@pytest.mark.parametrize("tau", [1.0, 0.45, 2.7])
def test_segments_of_every_shape(tau):
    rng = np.random.default_rng(int(tau * 100))
    lens = [0, 1, 2, 7, 2047, 2048, 2049, 65535, 65536, 65537, 131073, 200000, 5, 0, 300]
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(offsets[-1])
    logits = rng.normal(0.0, 3.0, n).astype(np.float32)
    mask = (rng.random(n) < 0.6).astype(np.uint8)
    logits[rng.random(n) < 0.05] = -np.inf            # masked by value as well
    ties = 0
    for counter in range(4):
        ties += _compare(logits, offsets, tau, 12345, counter, mask)
        ties += _compare(logits, offsets, tau, 999, counter, None)
    assert ties <= 2


def test_aligned_segments_with_ragged_parts():
    # segment starts on 16-logit boundaries: parts are staged by bulk copies,
    # with the last partial 16 bytes of logits and mask read directly
    rng = np.random.default_rng(5)
    lens = [16, 32, 8192, 8208, 16432, 1040, 8192 * 3 + 48, 64, 23]
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(offsets[-1])
    logits = rng.normal(0.0, 2.5, n).astype(np.float32)
    mask = (rng.random(n) < 0.5).astype(np.uint8)
    ties = 0
    for counter in range(6):
        ties += _compare(logits, offsets, 0.8, 77, counter, mask)
        ties += _compare(logits, offsets, 1.3, 78, counter, None)
    assert ties <= 2


def test_all_masked_and_single_entry():
    logits = np.array([1.0, 2.0, -np.inf, 5.0, 0.5, 0.25], np.float32)
    mask = np.array([0, 0, 1, 1, 0, 0], np.uint8)
    offsets = np.array([0, 2, 4, 6], np.int64)       # all masked / one admissible / all masked
    plan = SelectPlan(offsets)
    idx, logp = select_logits(plan, torch.from_numpy(logits).cuda(), 1.0, 3, 4, torch.from_numpy(mask).cuda())
    idx, logp = idx.cpu().numpy(), logp.cpu().numpy()
    assert idx.tolist() == [-1, 1, -1]
    assert math.isnan(logp[0]) and logp[1] == 0.0 and math.isnan(logp[2])
    with pytest.raises(AkmcError):
        select_logits(plan, torch.from_numpy(logits).cuda(), 0.0)
    with pytest.raises(AkmcError):
        SelectPlan(np.array([0, 5, 3], np.int64))     # decreasing offsets


def test_log_rates_reproduce_rejection_free_selection(model):
    # z = ln(Gamma) of real AKMC states, tau = 1: the draws follow Gamma / Gamma_tot
    descs = [synth.VoxelDesc(8, 6, (0.08, 0.06, 0.06), 563.0, synth.EAM_MODEL, synth.PREC_SPLIT, seed=40 + u, uid=u)
             for u in range(4)]
    b = Batch(descs, model)
    rates = [b.read_state(v)["rates"].ravel() for v in range(len(descs))]
    b.close()
    logits = np.concatenate([np.where(g > 0, np.log(np.where(g > 0, g, 1.0)), -np.inf) for g in rates])
    offsets = np.concatenate([[0], np.cumsum([g.size for g in rates])]).astype(np.int64)
    plan = SelectPlan(offsets)
    lt = torch.from_numpy(logits.astype(np.float32)).cuda()
    n = 4000
    counts = [np.zeros(g.size) for g in rates]
    for c in range(n):
        idx, _ = select_logits(plan, lt, 1.0, 2026, c)
        for s, j in enumerate(idx.cpu().numpy()):
            counts[s][j] += 1
    for s, g in enumerate(rates):
        p = g / g.sum()
        nz = p > 0
        assert counts[s][~nz].sum() == 0
        chi2 = float((((counts[s] - n * p) ** 2)[nz] / (n * p[nz])).sum())
        dof = int(nz.sum()) - 1
        assert chi2 < dof + 8 * math.sqrt(2 * dof), (s, chi2, dof)


def test_full_size_workload_sampled():
    # the benchmark shape: 256 systems of 65536 agents x 8 candidate transitions
    n_seg, per = 256, 65536 * 8
    rng = np.random.default_rng(7)
    logits = rng.normal(0.0, 2.0, n_seg * per).astype(np.float32)
    mask = (rng.random(n_seg * per) < 0.02).astype(np.uint8)
    offsets = (np.arange(n_seg + 1) * per).astype(np.int64)
    plan = SelectPlan(offsets)
    idx, logp = select_logits(plan, torch.from_numpy(logits).cuda(), 1.0, 5, 6, torch.from_numpy(mask).cuda())
    idx, logp = idx.cpu().numpy(), logp.cpu().numpy()
    for s in (0, 101, 255):
        b, e = offsets[s], offsets[s + 1]
        j, lp, margin = SEL.select_one(logits[b:e].astype(np.float64), SEL.uniform(5, 6, s), 1.0, mask[b:e])
        assert idx[s] == j or margin < TIE
        if idx[s] == j:
            assert abs(logp[s] - lp) <= 2e-5 + 1e-6 * abs(lp)
