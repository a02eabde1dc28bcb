"""Oracle pins for the dynamics (a5-a9): exact conservation, incremental vs
from-scratch rates, tree vs linear scan selection, pure-Fe analytic clock and
random walk, compensated clock vs exact summation, Boltzmann occupancy on a
tiny lattice, trapped/numeric stops, checkpoint/resume and Cu clusters
against a library connected-components routine."""
import copy
import math

import numpy as np
import pytest

import oracle
import synth

KB = synth.KB_EV


def _loaded(model, L, n_vac, fracs, seed, mdl, T=563.0, uid=None):
    d = synth.VoxelDesc(L, n_vac, (0, 0, 0), T, mdl, 0, seed=seed, uid=seed if uid is None else uid)
    v = oracle.Voxel(d, model)
    sp, vac = synth.random_lattice(L, n_vac, fracs, seed=seed)
    v.load(sp, vac)
    return v


@pytest.mark.parametrize("mdl,L", [(0, 4), (1, 5)])
def test_conservation_and_incremental_consistency(model, mdl, L):
    v = _loaded(model, L, 5, (0.12, 0.1, 0.1), 3 + mdl, mdl)
    before = np.bincount(v.state()["species"], minlength=5)
    v.set_debug(1 | 2 | 4)
    n = 1500 if mdl == 0 else 300
    for _ in range(4):
        v.step(n)
        assert v.status == oracle.OK
        s = v.state()
        assert np.array_equal(np.bincount(s["species"], minlength=5), before)
        assert (s["species"][s["vac_pos"]] == 4).all()
    c = v.debug_counts()
    assert c["checked"] == 4 * n
    assert c["rate_mismatch"] == 0 and c["rho_mismatch"] == 0
    assert c["scan_disagree"] == 0


def test_pure_fe_clock_and_walk(model):
    # Pure Fe, one vacancy: all 8 rates equal Gamma, Gamma_tot = 8 Gamma.
    # E[t_n] = n/(8 Gamma), Var = n/(8 Gamma)^2; the vacancy does an unbiased
    # walk: E|R|^2 = 3n half-units^2 and directions are uniform.
    T = 563.0
    gamma = 6e12 * math.exp(-0.62 / (KB * T))
    n = 100000
    sp = np.zeros(2 * 6 ** 3, np.uint8)
    sp[0] = 4
    v = oracle.Voxel(synth.VoxelDesc(6, 1, (0, 0, 0), T, 0, 0, seed=42, uid=7), model)
    v.load(sp, np.array([0], np.int32))
    log, dts = v.step(n, log=True, dt=True)
    s = v.state()
    t = s["t_hi"] + s["t_lo"]
    assert abs(t - n / (8 * gamma)) < 5 * math.sqrt(n) / (8 * gamma)
    assert np.allclose(dts.mean() * 8 * gamma, 1.0, atol=5 / math.sqrt(n))
    assert abs(dts.var() * (8 * gamma) ** 2 - 1.0) < 0.05
    counts = np.bincount(log % 8, minlength=8)
    chi2 = ((counts - n / 8) ** 2 / (n / 8)).sum()
    assert chi2 < 7 + 6 * math.sqrt(14)
    # unwrapped displacement equals the sum of hop vectors
    d = np.stack([np.where(log & 1, -1, 1), np.where(log & 2, -1, 1), np.where(log & 4, -1, 1)], 1)
    assert np.array_equal(d.sum(0), s["vac_disp"][0])
    # MSD over many independent walks
    r2 = []
    for u in range(200):
        w = oracle.Voxel(synth.VoxelDesc(6, 1, (0, 0, 0), T, 0, 0, seed=5, uid=u), model)
        w.load(sp, np.array([0], np.int32))
        w.step(400)
        r2.append((w.state()["vac_disp"][0] ** 2).sum())
    r2 = np.array(r2, dtype=np.float64)
    assert abs(r2.mean() - 3 * 400) < 5 * r2.std() / math.sqrt(len(r2))


def test_compensated_clock_matches_exact_sum(model):
    # Service-life start: at t ~ 1.5e9 s (about 48 years) one float64 ulp is
    # 2.4e-7 s, while dt ~ 7e-9 s; the (t_hi, t_lo) pair must still track the
    # exact sum of the increments.
    sp = np.zeros(2 * 4 ** 3, np.uint8)
    sp[5] = 4
    v = oracle.Voxel(synth.VoxelDesc(4, 1, (0, 0, 0), 563.0, 0, 0, seed=8, uid=8), model)
    t0 = 1.5e9
    v.load(sp, np.array([5], np.int32), t_hi=t0, t_lo=0.0)
    _, dts = v.step(20000, dt=True)
    s = v.state()
    exact = math.fsum(dts)
    got = (s["t_hi"] - t0) + s["t_lo"]
    assert abs(got - exact) <= 1e-6 * exact
    # plain addition stalls entirely at this magnitude
    plain = t0
    for x in dts[:100]:
        plain += x
    assert plain == t0
    # dt of each event is -ln(u2)/R with the event's own uniform
    R = v.total_rate()
    u2 = [oracle.event_uniforms(8, 8, k)[1] for k in range(5)]
    for k in range(5):
        assert dts[k] == -math.log(u2[k]) / R


def test_trapped_and_numeric_stops(model):
    # every site a vacancy: no admissible hop, the voxel is trapped before any event
    L = 3
    sp = np.full(2 * L ** 3, 4, np.uint8)
    v = oracle.Voxel(synth.VoxelDesc(L, 1, (0, 0, 0), 563.0, 0, 0, seed=1, uid=1), model)
    v.load(sp, np.arange(2 * L ** 3, dtype=np.int32))
    v.step(10)
    assert v.status == oracle.ETRAPPED and v.state()["n_events"] == 0
    # an embedding table too short for the lattice's densities flags a numeric error
    m = copy.deepcopy(model)
    m.F_tab = m.F_tab[:, :200, :].copy()      # covers rho < 0.39 only
    d = synth.VoxelDesc(4, 1, (0, 0, 0), 563.0, 1, 0, seed=2, uid=2)
    assert oracle.Voxel(d, m).status == oracle.ENUMERIC


def test_checkpoint_resume_is_bit_exact(model):
    for mdl, L in ((0, 5), (1, 5)):
        d = synth.VoxelDesc(L, 3, (0.05, 0.05, 0.05), 563.0, mdl, 0, seed=77, uid=4)
        a = oracle.Voxel(d, model)
        log_a = a.step(1200, log=True)
        b = oracle.Voxel(d, model)
        log_b1 = b.step(500, log=True)
        s = b.state()
        c = oracle.Voxel(d, model)
        c.load(s["species"], s["vac_pos"], s["t_hi"], s["t_lo"], s["n_events"])
        log_b2 = c.step(700, log=True)
        assert np.array_equal(log_a, np.concatenate([log_b1, log_b2]))
        sa, sc = a.state(), c.state()
        assert np.array_equal(sa["species"], sc["species"])
        assert sa["t_hi"] == sc["t_hi"] and sa["t_lo"] == sc["t_lo"]
        assert np.array_equal(sa["rates"], sc["rates"])


def _rel_class(L, vpos, cpos):
    def co(s):
        b, c = s & 1, s >> 1
        return np.array([2 * (c % L) + b, 2 * ((c // L) % L) + b, 2 * (c // (L * L)) + b])
    return tuple((co(cpos) - co(vpos)) % (2 * L))


@pytest.mark.slow
def test_boltzmann_occupancy_tiny_lattice(model):
    # L=3 pair model, one vacancy and one Cu in Fe (2862 states).  The chain
    # satisfies detailed balance, so the time-weighted occupancy of each
    # relative V-Cu configuration converges to exp(-E/kT)/Z, E by brute force.
    L, T = 3, 563.0
    beta = 1.0 / (KB * T)
    N = 2 * L ** 3
    sp = np.zeros(N, np.uint8)
    sp[0], sp[11] = 4, 1
    v = oracle.Voxel(synth.VoxelDesc(L, 1, (0, 0, 0), T, 0, 0, seed=2024, uid=1), model)
    v.load(sp, np.array([0], np.int32))
    n = 600000
    log, dts = v.step(n, log=True, dt=True)
    # replay positions (vacancy walks; Cu moves when it is the hop target)
    def co(s):
        b, c = s & 1, s >> 1
        return [2 * (c % L) + b, 2 * ((c // L) % L) + b, 2 * (c // (L * L)) + b]
    def site(X, Y, Z):
        M = 2 * L
        X, Y, Z = X % M, Y % M, Z % M
        return ((((Z >> 1) * L + (Y >> 1)) * L + (X >> 1)) << 1) | (X & 1)
    vpos, cpos = 0, 11
    keys = {}
    cls = np.empty(n, np.int32)
    for i, e in enumerate(log.tolist()):
        k = _rel_class(L, vpos, cpos)
        cls[i] = keys.setdefault(k, len(keys))
        X = co(vpos)
        m = site(X[0] + (-1 if e & 1 else 1), X[1] + (-1 if e & 2 else 1), X[2] + (-1 if e & 4 else 1))
        if m == cpos:
            cpos = vpos
        vpos = m
    # energies of each class (brute force), one representative each
    inv = {c: k for k, c in keys.items()}
    E = np.zeros(len(keys))
    for c, k in inv.items():
        X = np.array(k)
        s2 = np.zeros(N, np.uint8)
        s2[0] = 4
        s2[site(*X)] = 1
        w = oracle.Voxel(synth.VoxelDesc(L, 1, (0, 0, 0), T, 0, 0, seed=1, uid=1), model)
        w.load(s2, np.array([0], np.int32))
        E[c] = w.energy()
    assert len(keys) == N - 1
    p = np.exp(-beta * (E - E.min()))
    p /= p.sum()
    nb = 20
    fr = np.zeros((nb, len(keys)))
    for b in range(nb):
        sl = slice(b * n // nb, (b + 1) * n // nb)
        fr[b] = np.bincount(cls[sl], weights=dts[sl], minlength=len(keys)) / dts[sl].sum()
    mean, se = fr.mean(0), fr.std(0, ddof=1) / math.sqrt(nb)
    z = (mean - p) / np.maximum(se, 1e-4)
    assert np.abs(z).max() < 5.0
    assert np.abs(mean - p).sum() < 0.03


@pytest.mark.slow
def test_tracer_correlation_factor_bcc(model):
    # Pure Fe, one vacancy: sum over atoms of R_i^2 / (n * lambda^2) tends to
    # the bcc vacancy-mechanism correlation factor f = 0.7272 (textbook value).
    L, n = 8, 60000
    sp = np.zeros(2 * L ** 3, np.uint8)
    sp[0] = 4
    fs = []
    for u in range(6):
        v = oracle.Voxel(synth.VoxelDesc(L, 1, (0, 0, 0), 563.0, 0, 0, seed=31, uid=u), model)
        v.load(sp, np.array([0], np.int32))
        v.set_debug(8)
        v.step(n)
        fs.append(v.tracer_r2() / (n * 3.0))
    f = float(np.mean(fs))
    assert abs(f - 0.7272) < 0.02, fs


def test_cluster_histogram_matches_library_components(model):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    L = 6
    v = _loaded(model, L, 2, (0.12, 0.02, 0.02), 9, 0)
    sp = v.state()["species"]
    N = sp.size

    def co(s):
        b, c = s & 1, s >> 1
        return (2 * (c % L) + b, 2 * ((c // L) % L) + b, 2 * (c // (L * L)) + b)
    def site(X, Y, Z):
        M = 2 * L
        X, Y, Z = X % M, Y % M, Z % M
        return ((((Z >> 1) * L + (Y >> 1)) * L + (X >> 1)) << 1) | (X & 1)
    offs1 = [(a, b, c) for a in (-1, 1) for b in (-1, 1) for c in (-1, 1)]
    offs2 = [(2, 0, 0), (-2, 0, 0), (0, 2, 0), (0, -2, 0), (0, 0, 2), (0, 0, -2)]
    for mode, offs in ((0, offs1 + offs2), (1, offs1)):
        cu = np.flatnonzero(sp == 1)
        idx = {s: k for k, s in enumerate(cu)}
        rows, cols = [], []
        for s in cu:
            X = co(s)
            for o in offs:
                j = site(X[0] + o[0], X[1] + o[1], X[2] + o[2])
                if j in idx:
                    rows.append(idx[s])
                    cols.append(idx[j])
        g = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(len(cu), len(cu)))
        nc, lab = connected_components(g, directed=False)
        sizes = np.sort(np.bincount(lab))
        hist, got = v.cluster_hist(mode)
        assert np.array_equal(np.sort(got), sizes)
        bins = [0] * 8
        for s in sizes:
            bins[s - 1 if s <= 4 else (4 if s < 10 else (5 if s < 20 else (6 if s < 50 else 7)))] += 1
        assert hist.tolist() == bins
