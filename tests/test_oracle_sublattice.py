"""Oracle pins for the synchronous sublattice schedule (intra-voxel parallel
AKMC, the synchronous form of the sublattice scheme in Sec. 3.2.2): the
octants of one superstep are independent (any sector order gives the same
state, bit for bit), species are conserved, and in pure Fe the scheduled
vacancy walk has the analytic hop rate 8 Gamma per unit of voxel time and the
unbiased-walk mean squared displacement of 3 half-units^2 per hop."""
import math

import numpy as np
import pytest

import oracle
import synth

KB = synth.KB_EV


def _voxel(model, L, n_vac, fracs, seed, mdl, uid=None):
    d = synth.VoxelDesc(L, n_vac, (0, 0, 0), 563.0, mdl, 0, seed=seed, uid=seed if uid is None else uid)
    v = oracle.Voxel(d, model)
    sp, vac = synth.random_lattice(L, n_vac, fracs, seed=seed)
    v.load(sp, vac)
    return v


@pytest.mark.parametrize("mdl,L,S,nv", [(0, 20, 10, 12), (0, 16, 8, 20), (1, 16, 8, 8)])
def test_sector_order_independence(model, mdl, L, S, nv):
    # The events of one superstep's octants touch disjoint sets of sites, so
    # taking the sectors in reverse order must give the same lattice, the same
    # vacancy paths and the same event counts.
    a = _voxel(model, L, nv, (0.05, 0.03, 0.03), 11 + mdl, mdl)
    b = _voxel(model, L, nv, (0.05, 0.03, 0.03), 11 + mdl, mdl)
    T = 3.0 / (a.total_rate() / nv)
    ea = a.step_sublattice(0, 40, S, T)
    eb = b.step_sublattice(0, 40, S, T, reverse=True)
    sa, sb = a.state(), b.state()
    assert a.status == oracle.OK and b.status == oracle.OK
    assert ea.sum() > 20 * nv / 8
    assert np.array_equal(ea, eb)
    for k in ("species", "vac_pos", "vac_disp", "rates"):
        assert np.array_equal(sa[k], sb[k]), k
    assert sa["n_events"] == ea.sum()
    if mdl == 1:
        assert np.array_equal(a.rho_all(), b.rho_all())


@pytest.mark.parametrize("mdl", [0, 1])
def test_conservation_rates_and_clock(model, mdl):
    # Species counts are conserved, the incrementally refreshed rates equal a
    # from-scratch evaluation of the final lattice, and the clock advances by
    # exactly n_supersteps * T / 8.
    L, S, nv = 16, 8, 10
    v = _voxel(model, L, nv, (0.08, 0.05, 0.05), 5, mdl)
    before = np.bincount(v.state()["species"], minlength=5)
    T = 2.0 / (v.total_rate() / nv)
    n_st = 64
    ev = v.step_sublattice(3, n_st, S, T)
    s = v.state()
    assert v.status == oracle.OK
    assert np.array_equal(np.bincount(s["species"], minlength=5), before)
    assert (s["species"][s["vac_pos"]] == 4).all()
    w = oracle.Voxel(synth.VoxelDesc(L, nv, (0, 0, 0), 563.0, mdl, 0, seed=5, uid=5), model)
    w.load(s["species"], s["vac_pos"])
    assert np.array_equal(w.state()["rates"], s["rates"])
    assert s["t_hi"] + s["t_lo"] == pytest.approx(n_st * T / 8, rel=1e-15)
    assert s["n_events"] == ev.sum()


def test_invalid_sector_parameters(model):
    v = _voxel(model, 16, 2, (0, 0, 0), 1, 0)
    for S in (6, 7, 12, 32):
        with pytest.raises(ValueError):
            v.step_sublattice(0, 1, S, 1e-9)
    with pytest.raises(ValueError):
        v.step_sublattice(0, 1, 8, 0.0)


def test_pure_fe_scheduled_walk(model):
    # One vacancy in pure Fe: all 8 hop rates equal Gamma.  Over voxel time t
    # the scheduled walk makes 8 Gamma t hops on average (less a boundary loss
    # of about (8 Gamma T)(3/(2h))/2 for octants of h cells, here < 0.5 %), and
    # its squared displacement is 3 half-units^2 per hop.
    T = 563.0
    gamma = 6e12 * math.exp(-0.62 / (KB * T))
    L = S = 16
    win = 0.05 / (8 * gamma)
    n_st = 8 * 1500
    sp = np.zeros(2 * L ** 3, np.uint8)
    hops, r2 = [], []
    for u in range(160):
        site = int(np.random.default_rng(u).integers(0, 2 * L ** 3))
        sp[:] = 0
        sp[site] = 4
        v = oracle.Voxel(synth.VoxelDesc(L, 1, (0, 0, 0), T, 0, 0, seed=9, uid=u), model)
        v.load(sp, np.array([site], np.int32))
        ev = v.step_sublattice(0, n_st, S, win)
        s = v.state()
        hops.append(int(ev.sum()))
        r2.append(float((s["vac_disp"][0].astype(np.float64) ** 2).sum()))
    t = n_st * win / 8
    n = float(sum(hops))
    expect = 8 * gamma * t * len(hops)
    assert abs(n - expect) < 5 * math.sqrt(expect) + 0.005 * expect
    r2 = np.array(r2)
    h = np.array(hops, np.float64)
    # E|R|^2 = 3 n for an unbiased walk of n hops
    ratio = r2.sum() / (3 * h.sum())
    assert abs(ratio - 1.0) < 5 * r2.std() / math.sqrt(len(r2)) / (3 * h.mean())
