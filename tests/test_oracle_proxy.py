"""Pins of the oracle's Eq. 10 workload proxy (W = M exp(-E/kT), M the
admissible hops, E the effective barrier): closed forms in pure Fe, the
admissible-hop count by brute-force neighbour counting, the Jensen bounds
min Ea <= E <= mean Ea over the admissible hops, the temperature law of a
single-barrier state, and W = Gamma_tot / nu."""
import math

import numpy as np

import oracle
import synth
from oracle.proxy import KB_EV, workload_proxy


def _voxel(model, L, nv, frac, T, mdl=synth.PAIR_MODEL, seed=3, uid=1):
    return oracle.Voxel(synth.VoxelDesc(L, nv, frac, T, mdl, synth.PREC_FP64, seed=seed, uid=uid), model)


def test_pure_fe_closed_form(model):
    # single vacancies, or pair-model vacancies placed beyond each other's 2nn shell
    for T, nv, mdl in ((563.0, 1, synth.PAIR_MODEL), (543.0, 1, synth.EAM_MODEL), (593.0, 2, synth.PAIR_MODEL)):
        o = _voxel(model, 8, nv, (0.0, 0.0, 0.0), T, mdl)
        s = o.state()
        W, M, E = workload_proxy(s["rates"], T, model.nu)
        assert M == 8 * nv
        assert abs(E - model.E0[0]) <= 1e-12
        assert math.isclose(W, 8 * nv * math.exp(-model.E0[0] / (KB_EV * T)), rel_tol=1e-12)


def _nn1(L, site):
    c, b = divmod(site, 2)
    x, c = c % L, c // L
    y, z = c % L, c // L
    X, Y, Z = 2 * x + b, 2 * y + b, 2 * z + b
    out = []
    for dx in (-1, 1):
        for dy in (-1, 1):
            for dz in (-1, 1):
                Xn, Yn, Zn = (X + dx) % (2 * L), (Y + dy) % (2 * L), (Z + dz) % (2 * L)
                bn = Xn & 1
                out.append(((((Zn >> 1) * L + (Yn >> 1)) * L + (Xn >> 1)) << 1) | bn)
    return out


def test_admissible_hops_by_neighbour_count(model):
    # many vacancies, some of them 1nn neighbours: M = sum over vacancies of the
    # 1nn sites that are not vacancies (counted here from the lattice geometry)
    L = 4
    species, vac = synth.random_lattice(L, 40, (0.1, 0.1, 0.1), seed=7)
    d = synth.VoxelDesc(L, 40, (0.1, 0.1, 0.1), 563.0, synth.PAIR_MODEL, synth.PREC_FP64, seed=1, uid=1)
    o = oracle.Voxel(d, model)
    o.load(species, vac)
    s = o.state()
    M_brute = sum(sum(1 for j in _nn1(L, int(v)) if species[j] != synth.VAC) for v in vac)
    W, M, E = workload_proxy(s["rates"], 563.0, model.nu)
    assert M == M_brute < 8 * 40
    assert math.isclose(W * model.nu, o.total_rate(), rel_tol=1e-13)


def test_effective_barrier_jensen_bounds(model):
    beta = 1.0 / (KB_EV * 563.0)
    for mdl, frac in ((synth.PAIR_MODEL, (0.2, 0.1, 0.1)), (synth.EAM_MODEL, (0.1, 0.1, 0.05))):
        o = _voxel(model, 6, 4, frac, 563.0, mdl, seed=11)
        s = o.state()
        r = s["rates"].ravel()
        adm = r > 0
        Ea = -np.log(r[adm] / model.nu) / beta          # each admissible hop's barrier
        W, M, E = workload_proxy(r, 563.0, model.nu)
        assert Ea.min() - 1e-12 <= E <= Ea.mean() + 1e-12
        assert Ea.max() - Ea.min() > 0.01                # a real spread, so the bounds bite
        assert E < Ea.mean() - 1e-6


def test_single_barrier_temperature_law(model):
    # pure Fe: every hop has Ea = E0(Fe), so W(T1) / W(T2) = exp(-E0 (1/kT1 - 1/kT2))
    W1, _, _ = workload_proxy(_voxel(model, 6, 1, (0, 0, 0), 543.0).state()["rates"], 543.0, model.nu)
    W2, _, _ = workload_proxy(_voxel(model, 6, 1, (0, 0, 0), 593.0).state()["rates"], 593.0, model.nu)
    want = math.exp(-model.E0[0] * (1.0 / (KB_EV * 543.0) - 1.0 / (KB_EV * 593.0)))
    assert math.isclose(W1 / W2, want, rel_tol=1e-12)


def test_no_admissible_hop():
    W, M, E = workload_proxy(np.zeros(16), 563.0, 6e12)
    assert (W, M) == (0.0, 0) and E == math.inf
