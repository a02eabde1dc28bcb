"""TEST INFRASTRUCTURE ONLY: exact mean first-passage times of the vacancy
AKMC chain on a tiny state space (the Poisson equation of Eq. 5, the event
time increment of Eq. 6 and the dimensionless potential of Eq. 7).

States: one vacancy and one solute atom in an L^3-cell Fe lattice (from
synth.vacancy_solute_states).  Transitions: the 8 first-neighbour hops of the
vacancy with the oracle's rates; a hop onto the solute swaps the two.
tau(s) = 0 on the absorbing set A, and for s not in A
    sum_a Gamma_a(s) [tau(Phi(s, a)) - tau(s)] + 1 = 0                 (Eq. 5)
solved as a dense linear system in float64 (numpy).  Then
    delta_tau(s, a) = tau(s) - tau(Phi(s, a))                           (Eq. 6)
    u(s) = Gamma_tot(s) tau(s)                                          (Eq. 7)
Only tests/ use this module.
"""
from __future__ import annotations

import numpy as np

from . import Voxel


def half_coords(site: int, L: int):
    b, c = site & 1, site >> 1
    return np.array([2 * (c % L) + b, 2 * ((c // L) % L) + b, 2 * (c // (L * L)) + b])


def site_of(X, L: int) -> int:
    M = 2 * L
    X = [int(x) % M for x in X]
    return ((((X[2] >> 1) * L + (X[1] >> 1)) * L + (X[0] >> 1)) << 1) | (X[0] & 1)


def min_image_r2(a: int, b: int, L: int) -> int:
    """Squared minimal-image distance in half units (bcc shells 1..5: 3, 4, 8, 11, 12)."""
    d = half_coords(a, L) - half_coords(b, L)
    d = (d + L) % (2 * L) - L
    return int((d * d).sum())


def successors(vs, cs, L: int):
    """succ[s, d]: state index after hop d of the vacancy (dir = (dx<0)+2(dy<0)+4(dz<0))."""
    N = 2 * L ** 3
    index = {(int(v), int(c)): i for i, (v, c) in enumerate(zip(vs, cs))}
    succ = np.empty((vs.size, 8), np.int64)
    for i, (v, c) in enumerate(zip(vs, cs)):
        X = half_coords(int(v), L)
        for d in range(8):
            m = site_of(X + np.array([-1 if d & 1 else 1, -1 if d & 2 else 1, -1 if d & 4 else 1]), L)
            nv, nc = m, (int(v) if m == c else int(c))
            succ[i, d] = index[(nv, nc)]
    assert succ.max() < N * (N - 1)
    return succ


def oracle_rates(model, desc, species, vs):
    """Rates of the 8 hops of every state from the AKMC oracle (float64)."""
    out = np.empty((vs.size, 8))
    for i in range(vs.size):
        v = Voxel(desc, model)
        v.load(species[i], np.array([vs[i]], np.int32))
        out[i] = v.state()["rates"].ravel()
    return out


def solve_mfpt(rates, succ, absorbing):
    """tau(s) of Eq. 5 (zero on the absorbing set)."""
    n = rates.shape[0]
    tr = np.flatnonzero(~absorbing)
    pos = -np.ones(n, np.int64)
    pos[tr] = np.arange(tr.size)
    A = np.zeros((tr.size, tr.size))
    for r, s in enumerate(tr):
        A[r, r] += rates[s].sum()
        for d in range(8):
            t = succ[s, d]
            if not absorbing[t]:
                A[r, pos[t]] -= rates[s, d]
    tau = np.zeros(n)
    tau[tr] = np.linalg.solve(A, np.ones(tr.size))
    return tau


def delta_tau(tau, succ):
    return tau[:, None] - tau[succ]


def potential(tau, rates):
    return rates.sum(axis=1) * tau
