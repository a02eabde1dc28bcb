"""Temperature-guided voxel discretization (Sec. "Temperature-Guided
Discretization", Eq. 8-9).

The wall-thickness (r) and axial (z) extents of the vessel are cut uniformly
into n_r x n_z voxels.  Kinetic rates are Arrhenius, r(T) = r0 exp(-E / kB T)
(Eq. 8), so a temperature spread dT inside a voxel changes its rates by
dr / r ~ E dT / (kB T^2) (Eq. 9).  The counts are the smallest found, one
direction at a time, for which every voxel keeps that variation within a
tolerance (taken at the voxel's coolest point, where it is largest), so each
voxel can be simulated at one temperature.  The circumferential direction is
not cut (the service conditions are taken as homogeneous along it).

Host-side set-up, no device work: the result feeds the voxel descriptors
(one temperature per voxel) of a batch or a serving run.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Tuple

import numpy as np

KB_EV = 8.617333262e-5


def rate_variation(E: float, t_lo, t_hi):
    """First-order relative rate change E (t_hi - t_lo) / (kB t_lo^2) over a temperature range."""
    t_lo = np.asarray(t_lo, dtype=np.float64)
    return E * (np.asarray(t_hi, dtype=np.float64) - t_lo) / (KB_EV * t_lo * t_lo)


def _sample(T_of: Callable, wall: float, height: float, n_r: int, n_z: int, s: int) -> np.ndarray:
    """T on a grid with s points per voxel edge (shared between neighbours): shape (n_r(s-1)+1, n_z(s-1)+1)."""
    r = np.linspace(0.0, wall, n_r * (s - 1) + 1)
    z = np.linspace(0.0, height, n_z * (s - 1) + 1)
    R, Z = np.meshgrid(r, z, indexing="ij")
    t = np.asarray(T_of(R, Z), dtype=np.float64)
    t = np.broadcast_to(t, R.shape)
    if not np.all(np.isfinite(t)) or np.any(t <= 0):
        raise ValueError("temperatures must be finite and positive")
    return t


def _cells(t: np.ndarray, n_r: int, n_z: int, s: int) -> np.ndarray:
    """The samples of each voxel: shape (n_r, n_z, s, s)."""
    w = np.lib.stride_tricks.sliding_window_view(t, (s, s))
    return w[:: s - 1, :: s - 1][:n_r, :n_z]


def variations(T_of: Callable, wall: float, height: float, n_r: int, n_z: int, E: float,
               samples: int = 9) -> Tuple[float, float, float]:
    """Largest rate variation over any voxel (whole voxel, along r only, along z only)."""
    s = max(2, int(samples))
    c = _cells(_sample(T_of, wall, height, n_r, n_z, s), n_r, n_z, s)
    whole = rate_variation(E, c.min(axis=(2, 3)), c.max(axis=(2, 3))).max()
    along_r = rate_variation(E, c.min(axis=2), c.max(axis=2)).max()
    along_z = rate_variation(E, c.min(axis=3), c.max(axis=3)).max()
    return float(whole), float(along_r), float(along_z)


def temperature_guided_grid(T_of: Callable, wall: float, height: float, E: float, tol: float,
                            samples: int = 9, n_max: int = 4096) -> Tuple[int, int]:
    """Voxel counts (n_r, n_z): starting from one voxel, the count of the
    direction whose voxels show the larger rate variation grows by one until
    every voxel's variation E dT / (kB T^2) is at most `tol`.  For a field that
    varies along one direction only this is the smallest count that meets the
    tolerance there.  `T_of(r, z)` (kelvin) takes broadcastable arrays."""
    if not (E > 0 and tol > 0 and wall > 0 and height > 0):
        raise ValueError("E, tol, wall and height must be positive")
    n_r = n_z = 1
    while True:
        whole, vr, vz = variations(T_of, wall, height, n_r, n_z, E, samples)
        if whole <= tol:
            return n_r, n_z
        if vr >= vz:
            n_r += 1
        else:
            n_z += 1
        if n_r > n_max or n_z > n_max:
            raise ValueError("no grid of at most %d voxels per direction meets the tolerance" % n_max)


@dataclasses.dataclass
class VoxelSite:
    i: int          # index along the wall thickness
    j: int          # index along the axis
    r: float        # voxel centre
    z: float
    T: float        # temperature the voxel is simulated at (its centre)
    variation: float  # its rate variation E dT / (kB T^2)


def voxel_sites(T_of: Callable, wall: float, height: float, E: float, tol: float,
                samples: int = 9) -> List[VoxelSite]:
    """The voxels of the temperature-guided grid, row by row along r."""
    n_r, n_z = temperature_guided_grid(T_of, wall, height, E, tol, samples)
    s = max(2, int(samples))
    c = _cells(_sample(T_of, wall, height, n_r, n_z, s), n_r, n_z, s)
    var = rate_variation(E, c.min(axis=(2, 3)), c.max(axis=(2, 3)))
    out = []
    for i in range(n_r):
        for j in range(n_z):
            r = (i + 0.5) * wall / n_r
            z = (j + 0.5) * height / n_z
            T = float(np.asarray(T_of(np.float64(r), np.float64(z)), dtype=np.float64))
            out.append(VoxelSite(i, j, r, z, T, float(var[i, j])))
    return out
