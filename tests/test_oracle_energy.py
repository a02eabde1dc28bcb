"""Oracle pins for the energy model, barriers and rates (a2, a3, a4):
closed forms for pure Fe, exact Hermite reproduction of cubics, local hop
energy changes against brute-force full-lattice energy differences, and
detailed balance against brute-force energies (including the clamp branches)."""
import copy
import math

import numpy as np
import pytest

import oracle
import synth

KB = synth.KB_EV


def _voxel_from_lattice(model, L, n_vac, fracs, seed, mdl, T=563.0):
    d = synth.VoxelDesc(L, n_vac, (0.0, 0.0, 0.0), T, mdl, 0, seed=seed, uid=seed)
    v = oracle.Voxel(d, model)
    sp, vac = synth.random_lattice(L, n_vac, fracs, seed=seed)
    v.load(sp, vac)
    return v


def _pure_fe(model, L, mdl, T=563.0, vac_site=0):
    sp = np.zeros(2 * L ** 3, np.uint8)
    sp[vac_site] = 4
    d = synth.VoxelDesc(L, 1, (0.0, 0.0, 0.0), T, mdl, 0, seed=1, uid=1)
    v = oracle.Voxel(d, model)
    v.load(sp, np.array([vac_site], np.int32))
    return v


# ---------------------------------------------------------------- closed forms

def test_pair_energy_pure_fe_closed_form(model):
    L = 4
    N = 2 * L ** 3
    v = _pure_fe(model, L, 0)
    e1, e2 = model.eps1, model.eps2
    # bonds: N*8/2 first-shell, N*6/2 second-shell; those of the vacancy are Fe-V
    expect = (N * 4 - 8) * e1[0, 0] + 8 * e1[0, 4] + (N * 3 - 6) * e2[0, 0] + 6 * e2[0, 4]
    assert v.energy() == expect


def test_eam_energy_pure_fe_closed_form(model):
    L = 5
    N = 2 * L ** 3
    v = _pure_fe(model, L, 1, vac_site=17)
    phi, fq = oracle.shell_constants(model)
    counts = [8, 6, 12, 24, 8]
    rho0 = sum(c * f for c, f in zip(counts, fq[0]))
    Phi = sum(c * p for c, p in zip(counts, phi[0]))      # FeFe pair sum per atom
    F = lambda r: oracle.embed(model, 0, r)[0]
    expect = (N - 1 - 58) * F(rho0) + sum(c * F(rho0 - f) for c, f in zip(counts, fq[0]))
    expect += 0.5 * ((N - 1) * Phi - Phi)
    assert v.energy() == pytest.approx(expect, rel=1e-13, abs=1e-10)
    # density of an atom next to the vacancy is rho0 minus the 1nn contribution
    assert v.rho_fixed(17 ^ 1) in {rho0 - int(fq[0][k]) for k in range(5)} | {rho0}


def _poly_table(coef, n, h):
    x = np.arange(n) * h
    val = sum(c * x ** k for k, c in enumerate(coef))
    der = sum(k * c * x ** (k - 1) for k, c in enumerate(coef) if k)
    return np.stack([val, der], -1)


def test_shell_constants_reproduce_cubics(model):
    # Cubic Hermite interpolation is exact for cubics: shell values must equal
    # the polynomial at r_s = (a/2) sqrt(3, 4, 8, 11, 12).
    m = copy.deepcopy(model)
    dr = m.r_cut / (m.n_r - 1)
    pc = [0.7, -0.45, 0.08, -0.0041]
    fc = [0.3, -0.11, 0.012, -0.0004]
    m.phi_tab = np.stack([_poly_table(pc, m.n_r, dr)] * 10)
    m.f_tab = np.stack([_poly_table(fc, m.n_r, dr)] * 4)
    phi, fq = oracle.shell_constants(m)
    rs = m.a / 2 * np.sqrt([3, 4, 8, 11, 12])
    pv = sum(c * rs ** k for k, c in enumerate(pc))
    fv = sum(c * rs ** k for k, c in enumerate(fc))
    np.testing.assert_allclose(phi[3], pv, rtol=0, atol=1e-13)
    assert fq[2].tolist() == [int(math.floor(x * 2 ** 24 + 0.5)) for x in fv]


def test_embed_reproduces_cubic_and_flags_range(model):
    m = copy.deepcopy(model)
    cc = [-1.3, 0.8, -0.21, 0.033]
    m.F_tab = np.stack([_poly_table(cc, m.n_rho, m.rho_h)] * 4)
    for rf in (0, 1, 12345, 16777216, 23456789, 60000000):
        r = rf * 2.0 ** -24
        val, err = oracle.embed(m, 2, rf)
        assert err == 0
        assert val == pytest.approx(sum(c * r ** k for k, c in enumerate(cc)), abs=1e-13)
    top = (m.n_rho - 1) << 15   # last knot in fixed units (rho_h = 2^-9)
    assert oracle.embed(m, 0, top)[1] == 0
    assert oracle.embed(m, 0, top + 1)[1] == 1
    assert oracle.embed(m, 0, -1)[1] == 1


def test_rates_pure_fe_closed_form(model):
    # dE = 0 for every hop in pure Fe, Ea = E0(Fe) = 0.62 eV.
    for mdl, L in ((0, 4), (1, 5)):
        for T, expect in ((563.0, 1.690943e7), (543.0, None), (593.0, None)):
            v = _pure_fe(model, L, mdl, T=T)
            gamma = 6e12 * math.exp(-0.62 / (KB * T))
            if expect is not None:
                assert gamma == pytest.approx(expect, rel=1e-6)
            rates = v.state()["rates"][0]
            np.testing.assert_allclose(rates, gamma, rtol=1e-13)
            assert v.total_rate() == pytest.approx(8 * gamma, rel=1e-13)


# ---------------------------------------------------------------- local vs brute force

@pytest.mark.parametrize("L", [3, 4, 5])
@pytest.mark.parametrize("wild", [False, True])
def test_pair_local_de_equals_brute_force(model, wild_model, L, wild):
    m = wild_model if wild else model
    for seed in range(3):
        v = _voxel_from_lattice(m, L, 4, (0.15, 0.12, 0.1), seed + 10 * L, 0)
        for slot in range(4):
            for d in range(8):
                assert v.hop_de_local(slot, d) == v.hop_de_brute(slot, d)


@pytest.mark.parametrize("L", [4, 5])
def test_eam_local_de_equals_brute_force(model, L):
    worst = 0.0
    for seed in range(2):
        v = _voxel_from_lattice(model, L, 3, (0.12, 0.12, 0.12), seed + 7 * L, 1)
        for slot in range(3):
            for d in range(8):
                a, b = v.hop_de_local(slot, d), v.hop_de_brute(slot, d)
                worst = max(worst, abs(a - b))
    assert worst <= 1e-12


def test_eam_de_scale_is_moderate(model):
    # The synthetic potential is calibrated so typical |dE| stays below ~0.5 eV
    # in concentrated environments.
    des = []
    for seed in range(3):
        v = _voxel_from_lattice(model, 6, 4, (0.1, 0.1, 0.1), seed, 1)
        des += list(v.state()["dE"].ravel())
    des = np.abs(np.array(des))
    assert np.median(des) < 0.5 and des.max() < 2.0 and np.median(des) > 1e-3


# ---------------------------------------------------------------- detailed balance

def _reverse_rate(v, slot, d, model, mdl, L, T):
    """Rate of the reverse hop, on a fresh voxel loaded with the post-hop state."""
    s = v.state()
    sp = s["species"].copy()
    w = s["vac_pos"][slot]
    # post-hop lattice via the oracle's own step would also move the clock; build it directly
    X = _coords(w, L)
    dx, dy, dz = (-1 if d & 1 else 1, -1 if d & 2 else 1, -1 if d & 4 else 1)
    m = _site(L, X[0] + dx, X[1] + dy, X[2] + dz)
    sp[w], sp[m] = sp[m], 4
    pos = s["vac_pos"].copy()
    pos[slot] = m
    d2 = synth.VoxelDesc(L, len(pos), (0, 0, 0), T, mdl, 0, seed=3, uid=3)
    u = oracle.Voxel(d2, model)
    u.load(sp, pos)
    return u, u.hop_rate(slot, d ^ 7)


def _coords(s, L):
    b, c = s & 1, s >> 1
    return (2 * (c % L) + b, 2 * ((c // L) % L) + b, 2 * (c // (L * L)) + b)


def _site(L, X, Y, Z):
    M = 2 * L
    X, Y, Z = X % M, Y % M, Z % M
    return ((((Z >> 1) * L + (Y >> 1)) * L + (X >> 1)) << 1) | (X & 1)


@pytest.mark.parametrize("mdl,L", [(0, 4), (1, 4)])
@pytest.mark.parametrize("wild", [False, True])
def test_detailed_balance(model, wild_model, mdl, L, wild):
    m = wild_model if wild else model
    T = 563.0
    beta = 1.0 / (KB * T)
    clamp_hits = 0
    for seed in range(3):
        v = _voxel_from_lattice(m, L, 2, (0.15, 0.15, 0.1), 100 + seed, mdl, T)
        E_before = v.energy()
        for slot in range(2):
            for d in range(8):
                g_f = v.hop_rate(slot, d)
                if g_f == 0.0:
                    continue
                u, g_r = _reverse_rate(v, slot, d, m, mdl, L, T)
                # brute force: full-lattice energy difference (per-site differences summed
                # over every site for EAM, which keeps the float64 difference accurate)
                dE = u.energy() - E_before if mdl == 0 else v.hop_de_brute(slot, d)
                if mdl == 1:
                    assert abs((u.energy() - E_before) - dE) < 1e-10
                de_loc = v.hop_de_local(slot, d)
                A = v.state()["species"][_site(L, *[c + s for c, s in zip(
                    _coords(v.state()["vac_pos"][slot], L),
                    (-1 if d & 1 else 1, -1 if d & 2 else 1, -1 if d & 4 else 1))])]
                e0 = m.E0[A]
                if abs(de_loc) > 2 * e0:
                    clamp_hits += 1
                expect = math.exp(-dE * beta)
                assert g_f / g_r == pytest.approx(expect, rel=1e-12)
    if wild and mdl == 0:
        assert clamp_hits > 0   # the wild table exercises the clamped branches


def test_density_brute_force(model):
    """rho_i = sum over non-vacancy sites j within the cutoff of f_{s_j}(r_ij),
    by minimal-image distances over all site pairs (no stencil tables)."""
    L = 5
    v = _voxel_from_lattice(model, L, 3, (0.1, 0.1, 0.1), 41, 1)
    sp = v.state()["species"]
    N = sp.size
    s = np.arange(N)
    c = s >> 1
    b = s & 1
    X = np.stack([2 * (c % L) + b, 2 * ((c // L) % L) + b, 2 * (c // (L * L)) + b], -1)
    d = X[:, None, :] - X[None, :, :]
    d = (d + L) % (2 * L) - L                       # minimal image in half units
    r2 = (d ** 2).sum(-1)                           # (2 r / a)^2
    shell_r2 = {3: 0, 4: 1, 8: 2, 11: 3, 12: 4}     # bcc shells 1-5 in half units
    _, fq = oracle.shell_constants(model)
    rho = np.zeros(N, np.int64)
    for i in range(N):
        for j in range(N):
            k = shell_r2.get(int(r2[i, j]))
            if k is not None and sp[j] != 4:
                rho[i] += int(fq[sp[j]][k])
    np.testing.assert_array_equal(v.rho_all(), rho)
    assert all(v.rho_fixed(i) == rho[i] for i in range(0, N, 7))


def _hop_atoms(species, vac_pos, L):
    """Species at each vacancy's 8 first-neighbour hop targets (dir = (dx<0) + 2(dy<0) + 4(dz<0))."""
    out = np.zeros((len(vac_pos), 8), np.int64)
    for q, s in enumerate(vac_pos):
        b, c = s & 1, s >> 1
        X, Y, Z = 2 * (c % L) + b, 2 * ((c // L) % L) + b, 2 * (c // (L * L)) + b
        for d in range(8):
            dx, dy, dz = (-1 if d & 1 else 1), (-1 if d & 2 else 1), (-1 if d & 4 else 1)
            Xn, Yn, Zn = (X + dx) % (2 * L), (Y + dy) % (2 * L), (Z + dz) % (2 * L)
            out[q, d] = species[((((Zn >> 1) * L + (Yn >> 1)) * L + (Xn >> 1)) << 1) | (Xn & 1)]
    return out


@pytest.mark.parametrize("mdl", [0, 1])
def test_arrhenius_temperature_sensitivity(model, mdl):
    # Eq. 9: d ln(rate)/dT = Ea / (kB T^2) with Ea = max(0, dE, E0(A) + dE/2), checked by a
    # central difference of the rates of one alloy state at T (1 +- 1e-5).
    L, T, h = 6, 563.0, 563.0 * 1e-5
    sp, vac = synth.random_lattice(L, 4, (0.08, 0.05, 0.05), seed=23)
    rates = {}
    for Tx in (T - h, T, T + h):
        v = oracle.Voxel(synth.VoxelDesc(L, 4, (0, 0, 0), Tx, mdl, 0, seed=1, uid=1), model)
        v.load(sp, vac)
        st = v.state()
        rates[Tx] = st["rates"].reshape(-1, 8)
        if Tx == T:
            dE = st["dE"].reshape(-1, 8)
    A = _hop_atoms(sp, vac, L)
    E0 = np.asarray(model.E0)
    live = A != 4
    Ea = np.maximum(0.0, np.maximum(dE, E0[np.minimum(A, 3)] + dE / 2))
    slope = (np.log(rates[T + h][live]) - np.log(rates[T - h][live])) / (2 * h)
    np.testing.assert_allclose(slope, Ea[live] / (KB * T * T), rtol=1e-6)
    assert (rates[T][~live] == 0).all()
