"""EAM site densities on the GPU (akmc_read_density) against the oracle.

Densities are exact integers (unit 2^-24), so every comparison is bit-exact.
Covered: the strip kernel's 16-byte path (L % 8 == 0, aligned rows) and its
byte path (odd-sized voxels before it in the batch break the alignment, or
L % 8 != 0), strips narrower than 16 rows (L = 24, 40), z-chunked and whole-z
strips, the tile kernel for L > 256, densities after events (the step
kernel's incremental updates), and the full-size rate-kernel workload
(64^3-cell voxels, sampled voxels).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2604_24091_gb300 import Batch, AkmcError  # noqa: E402

E, P = synth.EAM_MODEL, synth.PAIR_MODEL


def _d(L, nv, frac, model=E, uid=0, prec=synth.PREC_SPLIT):
    return synth.VoxelDesc(L, nv, frac, 563.0, model, prec if model == E else synth.PREC_FP64,
                           synth.splitmix64(synth.SEED_BASE + 30, uid), uid)


def _check_all(b, descs, model, voxels):
    for v in voxels:
        o = oracle.Voxel(descs[v], model)
        st = b.read_state(v)
        o.load(st["species"], st["vac_pos"])
        np.testing.assert_array_equal(b.read_density(v).astype(np.int64), o.rho_all(), err_msg="voxel %d" % v)


def test_density_mixed_batch_all_paths(model):
    rich = (0.05, 0.05, 0.05)
    descs = [_d(8, 2, rich, uid=0),                # 16-byte path
             _d(5, 1, rich, model=P, uid=1),       # 250 species bytes: next rows unaligned
             _d(16, 3, rich, uid=2),               # byte path (unaligned), L % 8 == 0
             _d(24, 2, (0.01, 0.02, 0.02), uid=3),
             _d(6, 1, rich, uid=4),                # L % 8 != 0
             _d(10, 4, rich, uid=5),
             _d(5, 1, rich, uid=6),                # odd L: 1000 density bytes
             _d(40, 2, (0.003, 0.007, 0.014), uid=7),
             _d(32, 1, (0.003, 0.007, 0.014), uid=8)]
    b = Batch(descs, model)
    _check_all(b, descs, model, [i for i, d in enumerate(descs) if d.model == E])
    with pytest.raises(AkmcError):
        b.read_density(1)                          # pair-model voxel
    b.close()


def test_density_aligned_batch_whole_z(model):
    # 1024 strips of one 16-row strip each: whole-z strips (tz = L), all aligned
    descs = [_d(16, 1, (0.01, 0.02, 0.02), uid=u) for u in range(1024)]
    b = Batch(descs, model)
    _check_all(b, descs, model, [0, 1, 511, 1023])
    b.close()


def test_density_after_events_is_exact(model):
    descs = [_d(16, 4, (0.03, 0.03, 0.03), uid=10), _d(12, 2, (0.03, 0.03, 0.03), uid=11),
             _d(8, 1, (0.03, 0.03, 0.03), uid=12)]
    b = Batch(descs, model)
    b.step(np.array([20000, 20000, 20000], np.uint64))
    assert b.sync_status()[0] == 0
    _check_all(b, descs, model, [0, 1, 2])
    b.close()


def test_density_full_size_rate_workload(model):
    # the rate-kernel workload's voxels (64^3 cells, 2 vacancies), every site of
    # a few voxels; plus one 128^3-cell voxel (8-row strips)
    big = [synth.VoxelDesc(64, 2, (0.002, 0.01, 0.01), 563.0, E, synth.PREC_SPLIT, synth.splitmix64(99, u), u)
           for u in range(300)]
    b = Batch(big, model)
    _check_all(b, big, model, [0, 157, 299])
    b.close()
    huge = [synth.VoxelDesc(128, 64, (0.002, 0.007, 0.014), 563.0, E, synth.PREC_SPLIT, 5, 0)]
    b = Batch(huge, model)
    _check_all(b, huge, model, [0])
    b.close()


def test_density_tile_kernel_large_voxel(model):
    # L > 256 takes the tile kernel; sampled sites against the oracle's per-site density
    d = synth.VoxelDesc(260, 8, (0.002, 0.007, 0.014), 563.0, E, synth.PREC_SPLIT, 7, 3)
    b = Batch([d], model)
    rho = b.read_density(0)
    st = b.read_state(0)
    o = oracle.Voxel(d, model)
    o.load(st["species"], st["vac_pos"])
    rng = np.random.default_rng(1)
    sites = np.concatenate([rng.integers(0, rho.size, 20000), np.flatnonzero(st["species"] != 0)[:5000]])
    for s in sites:
        assert int(rho[s]) == o.rho_fixed(int(s)), s
    b.close()


def test_density_dense_lattices_overflow_path(model):
    # Locally dense lattices: more than 1024 non-Fe sites of one sublattice in a
    # block of 4 haloed planes sends the block through the direct scatter.
    descs = [_d(64, 4, (0.30, 0.30, 0.20), uid=25),    # 16-byte path, 80 % non-Fe
             _d(33, 2, (0.30, 0.30, 0.20), uid=26),    # byte path, 80 % non-Fe
             _d(64, 4, (0.10, 0.10, 0.10), uid=20),    # 16-byte path, ~30 % non-Fe
             _d(48, 4, (0.25, 0.15, 0.10), uid=21),    # 16-byte path, 16-row strips of 48 rows
             _d(33, 2, (0.30, 0.10, 0.10), uid=22),    # byte path
             _d(72, 3, (0.002, 0.01, 0.01), uid=23),   # 8-row strips, dilute
             _d(80, 3, (0.20, 0.10, 0.10), uid=24)]    # 8-row strips, dense
    b = Batch(descs, model)
    _check_all(b, descs, model, range(len(descs)))
    b.close()


def test_density_mixed_edges_and_dense_lattices(model):
    # voxels of several edges in one batch (16-byte path), dense ones overflowing the
    # per-block lists (direct scatter) in some or all blocks, z split in chunks; a
    # reset slot is rebuilt through the reset path's own strip list
    descs = [_d(64, 4, (0.10, 0.10, 0.10), uid=40),   # ~30 % non-Fe: lists overflow in some blocks
             _d(64, 4, (0.30, 0.30, 0.20), uid=41),   # 80 %: every block direct
             _d(48, 4, (0.25, 0.15, 0.10), uid=42),
             _d(72, 3, (0.002, 0.01, 0.01), uid=43),
             _d(80, 3, (0.20, 0.10, 0.10), uid=44),
             _d(8, 2, (0.05, 0.05, 0.05), uid=45),    # smallest: rows and planes wrap
             _d(16, 1, (0.05, 0.05, 0.05), uid=46),
             _d(24, 2, (0.01, 0.02, 0.02), uid=47)]
    b = Batch(descs, model)
    _check_all(b, descs, model, range(len(descs)))
    b.reset_voxels([3], [_d(72, 3, (0.004, 0.01, 0.01), uid=48)])
    descs[3] = _d(72, 3, (0.004, 0.01, 0.01), uid=48)
    _check_all(b, descs, model, [3])
    b.close()
