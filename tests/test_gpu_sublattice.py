"""GPU parity of the synchronous sublattice supersteps (one CTA per sector)
against the oracle's serial sector-by-sector schedule.

Bars: pair model and FP64 EAM bit-exact (lattice, vacancy positions and
displacements, event counts per superstep, clock); split-precision EAM by
conservation, exact densities and hop energy changes within 1e-5 eV on the
GPU's own lattice (its trajectory may leave the oracle's where two rates
differ within that tolerance).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2604_24091_gb300 import AkmcError, Batch, ETIMEOUT  # noqa: E402

SPLIT_DE_TOL = 1e-5


def _window(o, nv, per_vacancy_events):
    return per_vacancy_events / (o.total_rate() / nv)


def _compare_exact(b, v, o, per_step_g, per_step_o):
    g = b.read_state(v)
    so = o.state()
    assert np.array_equal(per_step_g, per_step_o)
    assert np.array_equal(g["species"], so["species"])
    assert np.array_equal(g["vac_pos"], so["vac_pos"])
    assert np.array_equal(g["vac_disp"], so["vac_disp"])
    assert g["n_events"] == so["n_events"]
    assert g["t_hi"] == so["t_hi"] and g["t_lo"] == so["t_lo"]
    np.testing.assert_allclose(g["rates"], so["rates"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("mdl,prec,L,Sc,nv", [(synth.PAIR_MODEL, synth.PREC_FP64, 16, 8, 12),
                                               (synth.PAIR_MODEL, synth.PREC_FP64, 24, 12, 30),
                                               (synth.EAM_MODEL, synth.PREC_FP64, 16, 8, 8)])
def test_supersteps_bit_exact(model, mdl, prec, L, Sc, nv):
    d = synth.VoxelDesc(L, nv, (0.06, 0.04, 0.04), 563.0, mdl, prec, seed=17 + L, uid=40 + nv)
    o = oracle.Voxel(d, model)
    T = _window(o, nv, 3.0)
    b = Batch([d], model)
    n_st = 24
    per_g = []
    for k in range(n_st):   # one call per superstep: per-superstep event counts
        before = b.read_state(0)["n_events"]
        b.step_sublattice(0, 5 + k, 1, Sc, T)
        per_g.append(b.read_state(0)["n_events"] - before)
    assert b.sync_status()[0] == 0
    per_o = o.step_sublattice(5, n_st, Sc, T)
    assert per_o.sum() > n_st * nv / 16
    _compare_exact(b, 0, o, np.array(per_g, np.uint64), per_o)
    b.close()


def test_many_supersteps_per_call_then_regular_steps(model):
    # 64 supersteps in one call, then ordinary events continue from the SL state
    d = synth.VoxelDesc(16, 10, (0.08, 0.05, 0.05), 563.0, synth.PAIR_MODEL, synth.PREC_FP64, seed=3, uid=9)
    o = oracle.Voxel(d, model)
    T = _window(o, 10, 2.0)
    b = Batch([d], model, event_log_capacity=4000)
    b.step_sublattice(0, 0, 64, 8, T)
    per_o = o.step_sublattice(0, 64, 8, T)
    g = b.read_state(0)
    assert g["n_events"] == per_o.sum()
    b.step(4000)
    log_o = o.step(4000, log=True)
    g = b.read_state(0, log=True)
    so = o.state()
    n0 = int(per_o.sum())
    order = (np.arange(4000) + n0) % 4000
    assert np.array_equal(g["event_log"][order], log_o)
    assert np.array_equal(g["species"], so["species"])
    assert np.array_equal(g["vac_disp"], so["vac_disp"])
    assert abs((g["t_hi"] + g["t_lo"]) - (so["t_hi"] + so["t_lo"])) <= 1e-12 * (so["t_hi"] + so["t_lo"])
    b.close()


def test_other_voxels_untouched_and_validation(model):
    P, F = synth.PAIR_MODEL, synth.PREC_FP64
    descs = [synth.VoxelDesc(8, 2, (0.05, 0, 0), 563.0, P, F, seed=1, uid=1),
             synth.VoxelDesc(16, 6, (0.05, 0, 0), 563.0, P, F, seed=2, uid=2)]
    b = Batch(descs, model)
    s0 = b.read_state(0)
    o = oracle.Voxel(descs[1], model)
    T = _window(o, 6, 2.0)
    b.step_sublattice(1, 0, 16, 8, T)
    per_o = o.step_sublattice(0, 16, 8, T)
    s1 = b.read_state(0)
    for k in ("species", "vac_pos", "rates"):
        assert np.array_equal(s0[k], s1[k])
    assert s1["n_events"] == 0 and s1["t_hi"] == 0.0
    assert b.read_state(1)["n_events"] == per_o.sum()
    for bad in [dict(voxel=2, sc=8, T=T), dict(voxel=1, sc=6, T=T), dict(voxel=1, sc=12, T=T),
                dict(voxel=0, sc=8, T=0.0), dict(voxel=1, sc=8, T=float("inf"))]:
        with pytest.raises(AkmcError):
            b.step_sublattice(bad["voxel"], 0, 1, bad["sc"], bad["T"])
    b.close()


def test_large_voxel_split_supersteps(model):
    # The large configuration (128^3 cells, 64 vacancies, EAM split) in sectors of
    # 16 cells: conservation, clock, exact densities and every hop energy change
    # within the split tolerance on the GPU's final lattice.
    d = synth.config_large()[0]
    b = Batch([d], model)
    o = oracle.Voxel(d, model)
    T = _window(o, d.n_vac, 4.0)
    b.step_sublattice(0, 0, 48, 16, T)
    assert b.sync_status()[0] == 0
    g = b.read_state(0)
    assert g["n_events"] > 48 * 64 / 8
    assert np.array_equal(np.bincount(g["species"], minlength=5), np.bincount(o.state()["species"], minlength=5))
    assert (g["species"][g["vac_pos"]] == 4).all()
    assert g["t_hi"] + g["t_lo"] == pytest.approx(48 * T / 8, rel=1e-15)
    o.load(g["species"], g["vac_pos"])
    np.testing.assert_array_equal(b.read_density(0).astype(np.int64), o.rho_all())
    so = o.state()
    assert np.abs(g["dE"] - so["dE"]).max() <= SPLIT_DE_TOL
    b.close()


def test_fp64_eam_larger_voxel_bit_exact(model):
    d = synth.VoxelDesc(32, 16, (0.003, 0.007, 0.014), 563.0, synth.EAM_MODEL, synth.PREC_FP64, seed=8, uid=12)
    o = oracle.Voxel(d, model)
    T = _window(o, 16, 6.0)
    b = Batch([d], model)
    b.step_sublattice(0, 0, 24, 16, T)
    per_o = o.step_sublattice(0, 24, 16, T)
    g = b.read_state(0)
    so = o.state()
    assert g["n_events"] == per_o.sum() > 24
    assert np.array_equal(g["species"], so["species"])
    assert np.array_equal(g["vac_disp"], so["vac_disp"])
    np.testing.assert_array_equal(b.read_density(0).astype(np.int64), o.rho_all())
    b.close()


@pytest.mark.parametrize("mdl,prec,L,Sc,nv", [(synth.PAIR_MODEL, synth.PREC_FP64, 16, 8, 12),
                                               (synth.PAIR_MODEL, synth.PREC_FP64, 24, 8, 30),
                                               (synth.PAIR_MODEL, synth.PREC_FP64, 32, 8, 256),
                                               (synth.EAM_MODEL, synth.PREC_FP64, 32, 8, 24)])
def test_async_readiness_matches_oracle(model, mdl, prec, L, Sc, nv):
    # one cooperative launch with per-sector readiness: the same result as the
    # synchronous schedule, bit for bit
    d = synth.VoxelDesc(L, nv, (0.06, 0.04, 0.04), 563.0, mdl, prec, seed=23 + L, uid=60 + nv)
    o = oracle.Voxel(d, model)
    T = _window(o, nv, 3.0)
    b = Batch([d], model)
    b.step_sublattice(0, 3, 40, Sc, T, asynchronous=True)
    b.step_sublattice(0, 43, 9, Sc, T, asynchronous=True)
    assert b.sync_status()[0] == 0
    per_o = o.step_sublattice(3, 49, Sc, T)
    g = b.read_state(0)
    so = o.state()
    assert g["n_events"] == so["n_events"] == per_o.sum() > 0
    assert np.array_equal(g["species"], so["species"])
    assert np.array_equal(g["vac_pos"], so["vac_pos"])
    assert np.array_equal(g["vac_disp"], so["vac_disp"])
    assert g["t_hi"] == so["t_hi"] and g["t_lo"] == so["t_lo"]
    np.testing.assert_allclose(g["rates"], so["rates"], rtol=1e-12, atol=0)
    if mdl == synth.EAM_MODEL:
        np.testing.assert_array_equal(b.read_density(0).astype(np.int64), o.rho_all())
    b.close()


@pytest.mark.parametrize("Sc", [8, 16])
def test_async_equals_sync_large_split(model, Sc):
    # the large configuration in split precision: both forms on the GPU agree
    # exactly (lattice, densities, vacancies, counters, clock)
    d = synth.config_large()[0]
    bs, ba = Batch([d], model), Batch([d], model)
    r = float(bs.read_state(0)["rates"].sum())
    T = 4.0 / (r / d.n_vac)
    bs.step_sublattice(0, 0, 64, Sc, T)
    ba.step_sublattice(0, 0, 64, Sc, T, asynchronous=True)
    assert bs.sync_status()[0] == 0 and ba.sync_status()[0] == 0
    gs, ga = bs.read_state(0), ba.read_state(0)
    assert gs["n_events"] == ga["n_events"] > 64 * 64 / 8
    for k in ("species", "vac_pos", "vac_disp"):
        assert np.array_equal(gs[k], ga[k]), k
    assert gs["t_hi"] == ga["t_hi"] and gs["t_lo"] == ga["t_lo"]
    assert np.array_equal(bs.read_density(0), ba.read_density(0))
    bs.close()
    ba.close()


def test_async_stalled_sector_times_out(model):
    # Failure detection without a fault: one sector never reports readiness, so
    # its neighbours' bounded waits run out; the voxel ends AKMC_ETIMEOUT, the
    # other voxel of the batch is untouched and the device stays usable.
    P, F = synth.PAIR_MODEL, synth.PREC_FP64
    descs = [synth.VoxelDesc(32, 8, (0.02, 0, 0), 563.0, P, F, seed=5, uid=1),
             synth.VoxelDesc(16, 4, (0.02, 0, 0), 563.0, P, F, seed=6, uid=2)]
    b = Batch(descs, model)
    o = oracle.Voxel(descs[0], model)
    T = _window(o, 8, 2.0)
    with pytest.raises(AkmcError):
        b.test_sublattice_stall(0, 4, 8, T, 64)            # sector index out of range
    before = b.read_state(1)
    b.test_sublattice_stall(0, 4, 8, T, 0)
    st, per = b.sync_status()
    assert per[0] == ETIMEOUT and per[1] == 0
    after = b.read_state(1)
    assert np.array_equal(before["species"], after["species"]) and after["n_events"] == 0
    b.close()
    # a fresh batch runs normally afterwards
    c = Batch([descs[0]], model)
    c.step_sublattice(0, 0, 16, 8, T, asynchronous=True)
    per_o = o.step_sublattice(0, 16, 8, T)
    g = c.read_state(0)
    assert c.sync_status()[0] == 0
    assert g["n_events"] == per_o.sum()
    assert np.array_equal(g["species"], o.state()["species"])
    c.close()
