"""Seeded synthetic inputs for the bcc Fe-Cu-Ni-Mn vacancy AKMC hot path.

This module is the one place where both the CUDA path and the oracle get their
inputs from.  It holds none of the method's arithmetic: it only draws model
parameter tables (pair energies, tabulated EAM functions) and voxel
descriptors from seeded generators, and it builds arbitrary test lattices.
Energy differences, barriers, rates, selection, time steps and observables
are computed separately by the oracle and by the kernels.

The paper (AtomWorld, arXiv 2604.24091) prints no interatomic model for the
classical AKMC baseline it accelerates, so the models here are synthetic:

* pair model: 1nn/2nn pair energies eps_k[a][b] drawn around a shell mean,
  rounded to multiples of 2^-24 eV so that every energy sum is exact in
  float64 (dyadic values), |eps| <= 0.8 eV;
* EAM: pair function phi_ab(r), density function f_b(r) (cubic splines in
  knot form sum_k c_k (r_k - r)^3 H(r_k - r), knots between the bcc shells,
  cutoff 5.6 A) and embedding function F_a(rho), each tabulated on a
  2000-point uniform grid as (value, derivative) pairs.  The tables *define*
  the potential: evaluation is cubic Hermite interpolation of the table.

Voxel workloads mirror the evaluated configurations (sizes, compositions,
temperatures, vacancy counts) with per-voxel seeds from splitmix64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# Species codes of the packed uint8 lattice.
FE, CU, NI, MN, VAC = 0, 1, 2, 3, 4
SPECIES = ("Fe", "Cu", "Ni", "Mn", "V")

KB_EV = 8.617333262e-5          # Boltzmann constant, eV/K (CODATA 2018)
LATTICE_A = 2.855               # bcc Fe lattice constant, Angstrom
R_CUT = 5.6                     # EAM cutoff, Angstrom (shells 1-5)
NU = 6.0e12                     # attempt frequency, 1/s
# Migration barrier of the jumping species at dE = 0 (eV): Fe, Cu given;
# Ni and Mn are builder choices without a literature claim.
E0 = (0.62, 0.56, 0.68, 0.64)

N_TABLE = 2000                  # points per tabulated EAM function
RHO_H = 2.0 ** -9               # knot spacing of F(rho); a power of two
SEED_BASE = 20260424

PAIR_MODEL, EAM_MODEL = 0, 1
PREC_FP64, PREC_SPLIT = 0, 1

_MASK64 = (1 << 64) - 1


def splitmix64(seed: int, uid: int) -> int:
    """Per-voxel 64-bit seed: splitmix64 (Vigna) finaliser of seed + (uid+1)*golden."""
    z = (seed + (uid + 1) * 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


# --------------------------------------------------------------------------
# Model parameters
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Model:
    """All energy-model inputs of one batch (both pair and EAM parts).

    eps1, eps2: float64 [5,5] symmetric pair energies of the 1st and 2nd
        neighbour shells, species order Fe, Cu, Ni, Mn, V (eV).
    E0: barrier of the jumping species at dE=0 (eV), order Fe, Cu, Ni, Mn.
    nu: attempt frequency (1/s).  a: lattice constant (A).
    phi_tab: float64 [10, n_r, 2] (value, d/dr) of phi_ab on r_k = k*r_cut/(n_r-1);
        pair index of a<=b is a*(7-a)/2 + b.
    f_tab: float64 [4, n_r, 2] (value, d/dr) of the density function f_b.
    F_tab: float64 [4, n_rho, 2] (value, d/drho) of F_a on rho_k = k*rho_h.
    """
    eps1: np.ndarray
    eps2: np.ndarray
    E0: Sequence[float] = E0
    nu: float = NU
    a: float = LATTICE_A
    r_cut: float = R_CUT
    phi_tab: Optional[np.ndarray] = None
    f_tab: Optional[np.ndarray] = None
    rho_h: float = RHO_H
    F_tab: Optional[np.ndarray] = None

    @property
    def n_r(self) -> int:
        return 0 if self.phi_tab is None else int(self.phi_tab.shape[1])

    @property
    def n_rho(self) -> int:
        return 0 if self.F_tab is None else int(self.F_tab.shape[1])


def pair_tables(seed: int = SEED_BASE, wild: bool = False):
    """1nn/2nn pair energies eps_k[a][b] = c_k + w*u (u ~ U[-1,1], symmetric),
    clipped to |eps| <= 0.8 eV and rounded to a multiple of 2^-24 eV.

    The default table uses w = 0.05 eV; the 'wild' table uses w = 0.8 eV so
    that barriers hit the clamps (negative and above-dE branches)."""
    rng = np.random.default_rng([seed, 0x5EED, int(wild)])
    c = (-0.60, -0.30)
    w = 0.8 if wild else 0.05
    out = []
    for k in range(2):
        e = np.zeros((5, 5))
        for i in range(5):
            for j in range(i, 5):
                v = c[k] + w * rng.uniform(-1.0, 1.0)
                v = min(0.8, max(-0.8, v))
                v = round(v * 2.0 ** 24) / 2.0 ** 24
                e[i, j] = e[j, i] = v
        out.append(e)
    return out[0], out[1]


_SPLINE_KNOTS = (2.6, 3.2, 4.2, 4.85, 5.6)   # between shells 1|2, 2|3, 3|4, 4|5, cutoff


def _shell_r(a: float) -> np.ndarray:
    return a * 0.5 * np.sqrt(np.array([3.0, 4.0, 8.0, 11.0, 12.0]))


def _knot_coeffs(targets: np.ndarray, a: float) -> np.ndarray:
    """Coefficients c_k of sum_k c_k (r_k - r)^3_+ hitting target values at the
    5 shell radii.  The basis matrix is triangular (knot k only reaches shells
    <= k), solved by numpy."""
    rs = _shell_r(a)
    B = np.array([[max(0.0, rk - r) ** 3 for rk in _SPLINE_KNOTS] for r in rs])
    return np.linalg.solve(B, targets)


def _tab_knot_spline(c: np.ndarray, n: int, r_cut: float) -> np.ndarray:
    r = np.arange(n, dtype=np.float64) * (r_cut / (n - 1))
    val = np.zeros(n)
    der = np.zeros(n)
    for ck, rk in zip(c, _SPLINE_KNOTS):
        d = np.maximum(0.0, rk - r)
        val += ck * d ** 3
        der += -3.0 * ck * d ** 2
    return np.stack([val, der], axis=-1)


def eam_tables(seed: int = SEED_BASE, n_r: int = N_TABLE, n_rho: int = N_TABLE,
               rho_h: float = RHO_H, a: float = LATTICE_A):
    """Seeded synthetic EAM: returns (phi_tab[10,n_r,2], f_tab[4,n_r,2], F_tab[4,n_rho,2]).

    Shell targets: f_Fe normalised so that the perfect-Fe density is ~1,
    solutes scaled by 1 +- 15 %; phi_FeFe attractive at 1nn/2nn, other
    pairs perturbed around it; F_a(rho) = -E_a sqrt(rho + 0.01) + G_a (rho-1)^2."""
    rng = np.random.default_rng([seed, 0xEA3])
    counts = np.array([8, 6, 12, 24, 8], dtype=np.float64)
    f_fe = np.array([30.63, 17.62, 3.81, 0.648, 0.2817])
    f_fe = f_fe / float(counts @ f_fe)
    f_tab = np.zeros((4, n_r, 2))
    for b in range(4):
        scale = 1.0 if b == FE else 1.0 + 0.15 * rng.uniform(-1.0, 1.0)
        tgt = f_fe * scale * (1.0 + 0.03 * rng.uniform(-1.0, 1.0, 5))
        f_tab[b] = _tab_knot_spline(_knot_coeffs(tgt, a), n_r, R_CUT)
    phi_fefe = np.array([-0.26, -0.11, 0.018, 0.008, -0.004])
    phi_tab = np.zeros((10, n_r, 2))
    for i in range(4):
        for j in range(i, 4):
            p = i * (7 - i) // 2 + j
            if i == FE and j == FE:
                tgt = phi_fefe.copy()
            else:
                tgt = phi_fefe * (1.0 + 0.25 * rng.uniform(-1.0, 1.0, 5)) \
                    + 0.02 * rng.uniform(-1.0, 1.0, 5) * np.array([1, 1, 0.3, 0.1, 0.1])
            phi_tab[p] = _tab_knot_spline(_knot_coeffs(tgt, a), n_r, R_CUT)
    F_tab = np.zeros((4, n_rho, 2))
    rho = np.arange(n_rho, dtype=np.float64) * rho_h
    for s in range(4):
        E = 3.0 * (1.0 if s == FE else 1.0 + 0.1 * rng.uniform(-1.0, 1.0))
        G = 0.5 * (1.0 if s == FE else 1.0 + 0.3 * rng.uniform(-1.0, 1.0))
        F_tab[s, :, 0] = -E * np.sqrt(rho + 0.01) + G * (rho - 1.0) ** 2
        F_tab[s, :, 1] = -0.5 * E / np.sqrt(rho + 0.01) + 2.0 * G * (rho - 1.0)
    return phi_tab, f_tab, F_tab


def default_model(seed: int = SEED_BASE, wild_pair: bool = False) -> Model:
    e1, e2 = pair_tables(seed, wild=wild_pair)
    phi, f, F = eam_tables(seed)
    return Model(eps1=e1, eps2=e2, phi_tab=phi, f_tab=f, F_tab=F)


# --------------------------------------------------------------------------
# Voxel descriptors
# --------------------------------------------------------------------------

@dataclasses.dataclass
class VoxelDesc:
    """One voxel: edge L (cells; 2L^3 sites), vacancy count, solute fractions
    of all sites (Cu, Ni, Mn; Fe is the balance), temperature (K), energy
    model (0 pair, 1 EAM), precision (0 FP64, 1 FP32/FP64 split), Philox
    seed and voxel uid (Philox counter word)."""
    L: int
    n_vac: int
    frac: Sequence[float]
    T: float
    model: int = PAIR_MODEL
    precision: int = PREC_FP64
    seed: int = 0
    uid: int = 0

    @property
    def n_sites(self) -> int:
        return 2 * self.L ** 3


def config_plain_pair() -> List[VoxelDesc]:
    """Plain AKMC, pair model: Fe-1.34at%Cu, 16^3 cells, 1 vacancy, 563 K, FP64."""
    s = SEED_BASE + 1
    return [VoxelDesc(16, 1, (0.0134, 0.0, 0.0), 563.0, PAIR_MODEL, PREC_FP64,
                      splitmix64(s, 0), 0)]


def config_batched_eam(n_voxels: int = 256, L: int = 32, precision: int = PREC_SPLIT,
                       T: float = 563.0) -> List[VoxelDesc]:
    """Batched EAM: n independent 32^3-cell voxels of Fe-0.3Cu-0.7Ni-1.4Mn at%,
    1 vacancy each."""
    s = SEED_BASE + 2
    return [VoxelDesc(L, 1, (0.003, 0.007, 0.014), T, EAM_MODEL, precision,
                      splitmix64(s, u), u) for u in range(n_voxels)]


def config_uneven(n_voxels: int = 1000, seed: int = SEED_BASE + 3) -> List[VoxelDesc]:
    """Uneven batch: L uniform in {16,24,32,48,64}, 1-8 vacancies, Cu 0.1-0.3,
    Ni/Mn 0.5-1.5 at%, T uniform in 543-593 K, pair/EAM mixed 50/50."""
    rng = np.random.default_rng([seed, 3])
    out = []
    for u in range(n_voxels):
        L = int(rng.choice([16, 24, 32, 48, 64]))
        nv = int(rng.integers(1, 9))
        cu = rng.uniform(0.001, 0.003)
        ni = rng.uniform(0.005, 0.015)
        mn = rng.uniform(0.005, 0.015)
        T = rng.uniform(543.0, 593.0)
        model = int(rng.integers(0, 2))
        prec = PREC_SPLIT if model == EAM_MODEL else PREC_FP64
        out.append(VoxelDesc(L, nv, (cu, ni, mn), T, model, prec, splitmix64(seed, u), u))
    return out


def config_large(L: int = 128, n_vac: int = 64) -> List[VoxelDesc]:
    """Large single voxel: 128^3 cells, Fe-0.2Cu-0.7Ni-1.4Mn at%, 64 vacancies, EAM split."""
    s = SEED_BASE + 4
    return [VoxelDesc(L, n_vac, (0.002, 0.007, 0.014), 563.0, EAM_MODEL, PREC_SPLIT,
                      splitmix64(s, 0), 0)]


def serving_requests(duration_s: float = 10.0, rate_hz: float = 200.0,
                     seed: int = SEED_BASE + 5, min_events: float = 1e6,
                     max_events: float = 1e7, precision: int = PREC_SPLIT):
    """Poisson arrivals of batched-EAM-like voxel requests.

    Returns a list of (arrival_time_s, VoxelDesc, n_events), events
    log-uniform in [min_events, max_events]."""
    rng = np.random.default_rng([seed, 5])
    t = 0.0
    out = []
    uid = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        n_ev = int(round(math.exp(rng.uniform(math.log(min_events), math.log(max_events)))))
        d = VoxelDesc(32, 1, (0.003, 0.007, 0.014), 563.0, EAM_MODEL, precision,
                      splitmix64(seed, uid), uid)
        out.append((t, d, n_ev))
        uid += 1
    return out


def mixed_requests(n: int, seed: int = SEED_BASE + 7, t_sim_range=(2e-4, 2e-3), sizes=(16, 24, 32),
                   max_vac: int = 2):
    """An ensemble of voxel requests of mixed shape, all due at once: edge L from
    `sizes`, 1..max_vac vacancies, pair or EAM (split precision) 50/50, Cu 0.1-0.3,
    Ni/Mn 0.5-1.5 at%, T uniform in 543-593 K, and a simulated-time horizon
    log-uniform in t_sim_range (seconds).  Returns (desc, t_sim) pairs."""
    rng = np.random.default_rng([seed, 7])
    out = []
    for u in range(n):
        L = int(rng.choice(sizes))
        nv = int(rng.integers(1, max_vac + 1))
        model = int(rng.integers(0, 2))
        prec = PREC_SPLIT if model == EAM_MODEL else PREC_FP64
        fr = (rng.uniform(0.001, 0.003), rng.uniform(0.005, 0.015), rng.uniform(0.005, 0.015))
        T = rng.uniform(543.0, 593.0)
        t_sim = float(math.exp(rng.uniform(math.log(t_sim_range[0]), math.log(t_sim_range[1]))))
        out.append((VoxelDesc(L, nv, fr, T, model, prec, splitmix64(seed, u), (1 << 40) + u), t_sim))
    return out


# --------------------------------------------------------------------------
# Arbitrary lattices for tests
# --------------------------------------------------------------------------

def random_lattice(L: int, n_vac: int, fracs=(0.1, 0.1, 0.1), seed: int = 0):
    """A random lattice with exact species counts (for loading arbitrary states).

    Returns (species uint8[2L^3], vac_pos int32[n_vac]); vacancy slots in the
    order drawn."""
    n = 2 * L ** 3
    rng = np.random.default_rng([seed, L, n_vac])
    perm = rng.permutation(n)
    species = np.zeros(n, dtype=np.uint8)
    vac = perm[:n_vac].astype(np.int32)
    species[vac] = VAC
    k = n_vac
    for s, fr in zip((CU, NI, MN), fracs):
        c = int(math.floor(fr * n + 0.5))
        species[perm[k:k + c]] = s
        k += c
    return species, vac


def precipitate_lattice(L: int, n_vac: int, cube: int = 4, fracs_ni_mn=(0.01, 0.01), seed: int = 0):
    """A lattice holding one compact Cu precipitate: every site of the cube of
    `cube`^3 cells at the origin is Cu (2*cube^3 sites); Ni, Mn and the
    vacancies are scattered at random over the rest.  Used to start ensembles
    far from equilibrium, so that the dynamics visibly moves the cluster
    histogram.  Returns (species uint8[2L^3], vac_pos int32[n_vac])."""
    n = 2 * L ** 3
    species = np.zeros(n, dtype=np.uint8)
    s = np.arange(n)
    c = s >> 1
    x, y, z = c % L, (c // L) % L, c // (L * L)
    in_cube = (x < cube) & (y < cube) & (z < cube)
    species[in_cube] = CU
    rest = np.flatnonzero(~in_cube)
    rng = np.random.default_rng([seed, L, n_vac, cube])
    perm = rng.permutation(rest)
    vac = perm[:n_vac].astype(np.int32)
    species[vac] = VAC
    k = n_vac
    for sp, fr in zip((NI, MN), fracs_ni_mn):
        cnt = int(math.floor(fr * n + 0.5))
        species[perm[k:k + cnt]] = sp
        k += cnt
    return species, vac


def vacancy_solute_states(L: int, solute: int = CU):
    """Every lattice of L^3 cells holding one vacancy and one solute atom in Fe:
    returns (vac_sites int32[n], solute_sites int32[n], species uint8[n, 2L^3]),
    n = N (N - 1) with N = 2L^3, ordered by (vacancy site, solute site)."""
    N = 2 * L ** 3
    vs, cs = [], []
    for v in range(N):
        for c in range(N):
            if c != v:
                vs.append(v)
                cs.append(c)
    vs = np.array(vs, np.int32)
    cs = np.array(cs, np.int32)
    sp = np.zeros((vs.size, N), np.uint8)
    sp[np.arange(vs.size), vs] = VAC
    sp[np.arange(vs.size), cs] = solute
    return vs, cs, sp
