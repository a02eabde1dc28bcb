"""Ensemble parity of the split-precision EAM path.

With FP32 embedding energies the GPU's rates differ from the float64 oracle's
by ~1e-6 relative, so individual trajectories eventually part; the
comparison is then statistical (the reading of the tolerance for the FP32
EAM variant): from one common far-from-equilibrium start (a compact Cu
precipitate, 128 Cu sites, in an L = 10 EAM voxel with 4 vacancies), 32 GPU
runs and 32 oracle runs with independent random streams take 20000 events
each; the mean Cu cluster-size histograms must agree within 2 standard errors
in every populated bin, one bin allowed to miss.  A power check requires that
the dissolution moved the monomer bin by more than 3 standard errors from its
start, so the test can tell a wrong dynamics (barriers, rates, selection)
from a right one.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

N_SEEDS = 32
N_EVENTS = 20000
L, NV, CUBE = 10, 4, 4


def _descs(uid0, precision):
    return [synth.VoxelDesc(L, NV, (0.0, 0.01, 0.01), 563.0, synth.EAM_MODEL, precision,
                            synth.splitmix64(synth.SEED_BASE + 20, u), u) for u in range(uid0, uid0 + N_SEEDS)]


def _zscores(a, b):
    se = np.sqrt(a.var(0, ddof=1) / len(a) + b.var(0, ddof=1) / len(b))
    diff = a.mean(0) - b.mean(0)
    populated = se > 0
    z = np.zeros_like(diff)
    z[populated] = diff[populated] / se[populated]
    assert np.all(diff[~populated] == 0), (a.mean(0), b.mean(0))
    return z


def test_split_eam_precipitate_dissolution_ensemble():
    model = synth.default_model()
    species, vac = synth.precipitate_lattice(L, NV, CUBE, seed=synth.SEED_BASE + 21)
    # the oracle first: its process pool is spawned before this process
    # touches the GPU
    h0_o, h1_o, st_o = oracle.ensemble_cluster_hist(_descs(1000, synth.PREC_FP64), model, N_EVENTS,
                                                    start=(species, vac))
    assert (st_o == 0).all()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2604_24091_gb300 import Batch
    b = Batch(_descs(0, synth.PREC_SPLIT), model)
    for v in range(N_SEEDS):
        b.load_state(v, species, vac)
    b.compute_rates()
    h0_g = np.array([b.cluster_hist(v) for v in range(N_SEEDS)])
    b.step(np.full(N_SEEDS, N_EVENTS, np.uint64))
    st, _ = b.sync_status()
    assert st == 0
    h1_g = np.array([b.cluster_hist(v) for v in range(N_SEEDS)])
    b.close()
    assert (h0_g == h0_o).all()                     # same start, exact histograms
    assert h0_o[0].tolist() == [0, 0, 0, 0, 0, 0, 0, 1]
    z_move = _zscores(h1_o, h0_o)
    assert z_move[0] > 3, z_move                    # power: monomers appeared
    z = _zscores(h1_g, h1_o)
    assert (np.abs(z) > 2).sum() <= 1, (z, h1_g.mean(0), h1_o.mean(0))
