"""Oracle pins: Philox4x32-10 (published known answers), the uniform mapping,
and the seeded placement of species (a1)."""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, expect in rows:
        assert oracle.philox4x32_10(ctr, key) == expect


def test_uniform_mapping_bits_and_range():
    # u1 = 53 bits (x0 << 21 | x1 >> 11) * 2^-53 in [0,1); u2 = (same from x2,x3) + 1 ulp, in (0,1].
    seed, uid = 0x0123456789ABCDEF, 0xFEDCBA9876543210
    for n in (0, 1, 2, 1 << 32, (1 << 40) + 7):
        u1, u2 = oracle.event_uniforms(seed, uid, n)
        ctr = [n & 0xFFFFFFFF, n >> 32, uid & 0xFFFFFFFF, (uid >> 32) & 0x7FFFFFFF]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        x = oracle.philox4x32_10(ctr, key)
        a = (x[0] << 21) | (x[1] >> 11)
        b = (x[2] << 21) | (x[3] >> 11)
        assert u1 == a * 2.0 ** -53 and 0.0 <= u1 < 1.0
        assert u2 == (b + 1) * 2.0 ** -53 and 0.0 < u2 <= 1.0


def test_uniforms_moments():
    u = np.array([oracle.event_uniforms(7, 3, n) for n in range(20000)])
    for col in range(2):
        assert abs(u[:, col].mean() - 0.5) < 5 * math.sqrt(1 / 12 / len(u))
        assert abs(u[:, col].var() - 1 / 12) < 0.005
    assert abs(np.corrcoef(u[:, 0], u[:, 1])[0, 1]) < 0.05


def _counts(desc):
    N = desc.n_sites
    return [int(math.floor(f * N + 0.5)) for f in desc.frac]


def test_placement_counts_and_slots(model):
    # 256 x 65536 sites at Fe-0.3Cu-0.7Ni-1.4Mn: 917.5 Mn rounds up (+0.5 floor rule).
    d = synth.config_batched_eam(1)[0]
    assert _counts(d) == [197, 459, 918]
    v = oracle.Voxel(d, model)
    s = v.state()
    assert np.bincount(s["species"], minlength=5).tolist() == [65536 - 1 - 197 - 459 - 918, 197, 459, 918, 1]
    assert s["species"][s["vac_pos"]].tolist() == [4]
    # plain config: 8192 * 0.0134 = 109.77 -> 110 Cu
    d1 = synth.config_plain_pair()[0]
    s1 = oracle.Voxel(d1, model).state()
    assert (s1["species"] == 1).sum() == 110


def test_placement_is_deterministic_and_seed_dependent(model):
    d = synth.VoxelDesc(6, 3, (0.05, 0.05, 0.05), 563.0, 0, 0, seed=11, uid=5)
    a = oracle.Voxel(d, model).state()["species"]
    b = oracle.Voxel(d, model).state()["species"]
    assert np.array_equal(a, b)
    d2 = synth.VoxelDesc(6, 3, (0.05, 0.05, 0.05), 563.0, 0, 0, seed=12, uid=5)
    assert not np.array_equal(a, oracle.Voxel(d2, model).state()["species"])


def test_placement_uniform_over_sites(model):
    # Every site is equally likely to receive the vacancy: chi-square over 54 sites.
    N = 54
    hits = np.zeros(N)
    trials = 5400
    for u in range(trials):
        d = synth.VoxelDesc(3, 1, (0.0, 0.0, 0.0), 563.0, 0, 0, seed=99, uid=u)
        hits[oracle.Voxel(d, model).state()["vac_pos"][0]] += 1
    exp = trials / N
    chi2 = ((hits - exp) ** 2 / exp).sum()
    # 53 degrees of freedom: mean 53, sd ~10.3; reject beyond ~5 sd
    assert chi2 < 53 + 5 * math.sqrt(2 * 53)


def test_invalid_descriptors(model):
    with pytest.raises(ValueError):
        oracle.Voxel(synth.VoxelDesc(2, 1, (0, 0, 0), 563.0, 0), model)     # pair needs L >= 3
    with pytest.raises(ValueError):
        oracle.Voxel(synth.VoxelDesc(3, 1, (0, 0, 0), 563.0, 1), model)     # EAM needs L >= 4
    with pytest.raises(ValueError):
        oracle.Voxel(synth.VoxelDesc(3, 1, (0.6, 0.6, 0.0), 563.0, 0), model)  # over-full
    with pytest.raises(ValueError):
        oracle.Voxel(synth.VoxelDesc(3, 0, (0.1, 0, 0), 563.0, 0), model)   # no vacancy
