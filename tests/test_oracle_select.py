"""Pins of the float64 reference of the logit-form global selection (Eq. 1-2):
closed forms (softmax of log-rates, equal logits, one admissible entry, two
entries at any temperature), agreement with the rejection-free linear scan of
the AKMC oracle at z = ln(Gamma), tau = 1, and frequencies of many draws."""
import math

import numpy as np
import pytest

import oracle
import oracle.select as SEL
import synth


def test_softmax_of_log_rates_is_rate_fraction(model):
    d = synth.VoxelDesc(6, 5, (0.08, 0.06, 0.06), 563.0, synth.PAIR_MODEL, 0, seed=11, uid=11)
    g = oracle.Voxel(d, model).state()["rates"].ravel()
    z = np.where(g > 0, np.log(np.where(g > 0, g, 1.0)), -np.inf)
    p, ok = SEL.softmax_probs(z, 1.0)
    np.testing.assert_allclose(p, g / g.sum(), rtol=1e-12, atol=0)
    assert np.array_equal(ok, g > 0)


def test_equal_logits_closed_form():
    z = np.full(10, 2.5)
    mask = np.array([1, 0, 1, 1, 0, 1, 1, 1, 0, 1], np.uint8)
    adm = np.flatnonzero(mask)
    for u in (0.0, 0.13, 0.5, 0.999):
        j, logp, _ = SEL.select_one(z, u, 1.7, mask)
        assert j == adm[int(math.floor(u * adm.size))]
        assert logp == pytest.approx(-math.log(adm.size), abs=1e-12)


def test_single_admissible_entry_and_none():
    z = np.array([-np.inf, 3.0, -np.inf, np.nan])
    for u in (0.0, 0.7):
        j, logp, _ = SEL.select_one(z, u)
        assert j == 1 and logp == 0.0
    j, logp, _ = SEL.select_one(np.array([-np.inf, -np.inf]), 0.3)
    assert j == -1 and math.isnan(logp)


def test_two_entries_any_temperature():
    z1, z2 = 0.7, -1.9
    for tau in (0.25, 1.0, 3.5):
        p, _ = SEL.softmax_probs([z1, z2], tau)
        p1 = 1.0 / (1.0 + math.exp((z2 - z1) / tau))
        assert p[0] == pytest.approx(p1, rel=1e-14)
        j, _, _ = SEL.select_one([z1, z2], p1 * (1 - 1e-9), tau)
        assert j == 0
        j, _, _ = SEL.select_one([z1, z2], p1 * (1 + 1e-9), tau)
        assert j == 1


def test_matches_rejection_free_scan(model):
    # z = ln(Gamma), tau = 1 selects the event of the linear scan
    # sum_{i <= j} Gamma_i > u Gamma_tot, except within rounding of a boundary
    d = synth.VoxelDesc(7, 6, (0.08, 0.06, 0.06), 563.0, synth.EAM_MODEL, 0, seed=12, uid=12)
    g = oracle.Voxel(d, model).state()["rates"].ravel()
    z = np.where(g > 0, np.log(np.where(g > 0, g, 1.0)), -np.inf)
    c = np.cumsum(g)
    rng = np.random.default_rng(5)
    ties = 0
    for u in rng.random(2000):
        j, _, margin = SEL.select_one(z, u)
        k = int(np.searchsorted(c, u * c[-1], side="right"))
        if margin < 1e-12:
            ties += 1
            continue
        assert j == k
    assert ties == 0


def test_draw_frequencies():
    z = np.array([0.3, -1.2, 2.0, -np.inf, 0.9, 1.1])
    p, _ = SEL.softmax_probs(z, 1.3)
    n = 20000
    counts = np.zeros(z.size)
    for c in range(n):
        j, _, _ = SEL.select_one(z, SEL.uniform(77, c, 0), 1.3)
        counts[j] += 1
    nz = p > 0
    chi2 = float((((counts - n * p) ** 2)[nz] / (n * p[nz])).sum())
    assert counts[3] == 0
    assert chi2 < 30.0, chi2          # 4 degrees of freedom; p(chi2 > 30) ~ 5e-6
    us = [SEL.uniform(1, c, 0) for c in range(1000)]
    assert min(us) >= 0.0 and max(us) < 1.0
