"""Temperature-guided voxel discretization (Sec. "Temperature-Guided
Discretization", Eq. 8-9) against closed forms and brute force."""
import math

import numpy as np
import pytest

from paper_2604_24091_gb300 import voxelize as V

KB = V.KB_EV
E = 0.6


def test_isothermal_vessel_is_one_voxel():
    n = V.temperature_guided_grid(lambda r, z: 563.0 + 0 * r, 0.2, 1.0, E, 0.01)
    assert n == (1, 1)
    sites = V.voxel_sites(lambda r, z: 563.0 + 0 * r, 0.2, 1.0, E, 0.01)
    assert len(sites) == 1 and sites[0].T == 563.0 and sites[0].variation == 0.0


def test_linear_wall_profile_closed_form():
    # T falls linearly by 30 K across the wall: the coolest voxel carries the
    # largest variation E (30/n) / (kB 533^2), so n is the smallest integer with
    # that at most tol; nothing varies axially.
    wall, tol = 0.2, 0.05
    T = lambda r, z: 563.0 - 30.0 * r / wall + 0 * z
    n_r, n_z = V.temperature_guided_grid(T, wall, 3.0, E, tol)
    expect = math.ceil(E * 30.0 / (KB * 533.0 ** 2 * tol))
    assert (n_r, n_z) == (expect, 1)
    assert E * (30.0 / (n_r - 1)) / (KB * 533.0 ** 2) > tol


def test_axial_profile_smallest_count_by_brute_force():
    height, tol = 4.0, 0.02
    T = lambda r, z: 543.0 + 40.0 * (z / height) ** 2 + 0 * r
    n_r, n_z = V.temperature_guided_grid(T, 0.2, height, E, tol, samples=33)

    def worst(n):   # the field rises along z: each voxel spans [T(z0), T(z1)]
        z = np.linspace(0.0, height, n + 1)
        t = 543.0 + 40.0 * (z / height) ** 2
        return max(E * (t[k + 1] - t[k]) / (KB * t[k] ** 2) for k in range(n))

    smallest = next(n for n in range(1, 1000) if worst(n) <= tol)
    assert n_r == 1 and n_z == smallest


def test_two_dimensional_field_every_voxel_within_tolerance():
    wall, height, tol = 0.25, 5.0, 0.03
    T = lambda r, z: 570.0 - 25.0 * r / wall + 15.0 * np.sin(np.pi * z / height)
    sites = V.voxel_sites(T, wall, height, E, tol)
    n_r = max(s.i for s in sites) + 1
    n_z = max(s.j for s in sites) + 1
    assert len(sites) == n_r * n_z and n_r > 1 and n_z > 1
    assert max(s.variation for s in sites) <= tol
    # an independent dense check of every voxel
    for s in sites:
        r = np.linspace(s.i * wall / n_r, (s.i + 1) * wall / n_r, 41)
        z = np.linspace(s.j * height / n_z, (s.j + 1) * height / n_z, 41)
        t = T(*np.meshgrid(r, z, indexing="ij"))
        assert E * (t.max() - t.min()) / (KB * t.min() ** 2) <= tol * (1 + 1e-3)
        assert s.T == pytest.approx(T(s.r, s.z))


def test_rejects_bad_input():
    with pytest.raises(ValueError):
        V.temperature_guided_grid(lambda r, z: 563.0 + 0 * r, 0.2, 1.0, E, 0.0)
    with pytest.raises(ValueError):
        V.temperature_guided_grid(lambda r, z: -1.0 + 0 * r, 0.2, 1.0, E, 0.1)
