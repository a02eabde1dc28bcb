"""TEST INFRASTRUCTURE ONLY: the workload proxy of the dynamic voxel
scheduling (Sec. "Dynamic Voxel Scheduling", Eq. 10) from an oracle voxel's
hop rates.

Eq. 10 gives W_v ~ M_v exp(-E_v / (kB T_v)), M_v a multiplicity of local
events and E_v an effective barrier set by the voxel's defect state.
Reading taken: M = the number of admissible hops (rate > 0) of all the
voxel's vacancies, and E the single barrier that gives each of them the
voxel's mean rate, E = -kB T ln(Gamma_tot / (nu M)), so that
W = M exp(-E / (kB T)) = Gamma_tot / nu.  Plain float64 (math.fsum for the
rate sum)."""
from __future__ import annotations

import math

import numpy as np

KB_EV = 8.617333262e-5


def workload_proxy(rates, T, nu):
    """(W, M, E) of one voxel from its 8 n_vac hop rates (any shape)."""
    r = np.asarray(rates, dtype=np.float64).ravel()
    M = int(np.count_nonzero(r > 0.0))
    G = math.fsum(r.tolist())
    W = G / nu
    E = -KB_EV * T * math.log(W / M) if (M > 0 and G > 0.0) else math.inf
    return W, M, E
