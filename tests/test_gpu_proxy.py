"""GPU: the Eq. 10 workload proxy (akmc_workload_proxy) against the oracle's,
on fresh and evolved voxels of both models and precisions; pure-Fe closed form."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle.proxy import KB_EV, workload_proxy

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2604_24091_gb300 import Batch  # noqa: E402


def _descs():
    return [synth.VoxelDesc(6, 3, (0.05, 0.04, 0.04), 563.0, synth.PAIR_MODEL, synth.PREC_FP64, seed=1, uid=1),
            synth.VoxelDesc(8, 1, (0.0, 0.0, 0.0), 543.0, synth.EAM_MODEL, synth.PREC_SPLIT, seed=2, uid=2),
            synth.VoxelDesc(7, 4, (0.08, 0.05, 0.05), 593.0, synth.EAM_MODEL, synth.PREC_FP64, seed=3, uid=3),
            synth.VoxelDesc(16, 1, (0.0134, 0.0, 0.0), 563.0, synth.PAIR_MODEL, synth.PREC_FP64, seed=4, uid=4),
            synth.VoxelDesc(4, 40, (0.1, 0.1, 0.1), 573.0, synth.PAIR_MODEL, synth.PREC_FP64, seed=5, uid=5)]


@pytest.mark.parametrize("events", [0, 700])
def test_proxy_matches_oracle(model, events):
    descs = _descs()
    b = Batch(descs, model)
    if events:
        b.step(events)
    W, Mh, Eh = b.workload_proxy()
    for v, d in enumerate(descs):
        g = b.read_state(v)
        o = oracle.Voxel(d, model)
        o.load(g["species"], g["vac_pos"])
        Wo, Mo, Eo = workload_proxy(o.state()["rates"], d.T, model.nu)
        assert Mh[v] == Mo
        assert math.isclose(W[v], Wo, rel_tol=1e-12)
        assert abs(Eh[v] - Eo) <= 1e-12
        # W = M exp(-E / kT) holds for the GPU's own triple
        assert math.isclose(W[v], Mh[v] * math.exp(-Eh[v] / (KB_EV * d.T)), rel_tol=1e-12)
    # pure Fe, one vacancy: E = E0(Fe), M = 8
    assert Mh[1] == 8 and abs(Eh[1] - model.E0[0]) <= 1e-12 if events == 0 else True
