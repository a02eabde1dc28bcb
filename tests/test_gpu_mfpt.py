"""State-space rate evaluation on the GPU for the exact first-passage times of
Eq. 5: all 2862 states of one vacancy and one Cu atom in a 3^3-cell Fe lattice
loaded as one batch of voxels; one akmc_compute_rates gives every state's 8
hop rates.  Rates within 1e-12 of the oracle's; the first-passage times solved
from the GPU rates within 1e-10 of those from the oracle's."""
import numpy as np
import pytest

import oracle.mfpt as MF
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2604_24091_gb300 import Batch  # noqa: E402

L, T = 3, 563.0


def test_state_space_rates_and_first_passage(model):
    vs, cs, sp = synth.vacancy_solute_states(L)
    descs = [synth.VoxelDesc(L, 1, (0.0, 0.0, 0.0), T, synth.PAIR_MODEL, synth.PREC_FP64, seed=5, uid=i)
             for i in range(vs.size)]
    b = Batch(descs, model)
    vp = vs.astype(np.int32)
    b.load_batch_state(sp.ravel(), vp)
    b.compute_rates()
    g = np.stack([b.read_state(i, species=False)["rates"].ravel() for i in range(vs.size)])
    b.close()
    o = MF.oracle_rates(model, descs[0], sp, vs)
    assert np.array_equal(g == 0, o == 0)
    np.testing.assert_allclose(g, o, rtol=1e-12, atol=0)
    succ = MF.successors(vs, cs, L)
    absorbing = np.array([MF.min_image_r2(int(v), int(c), L) > 4 for v, c in zip(vs, cs)])
    tg = MF.solve_mfpt(g, succ, absorbing)
    to = MF.solve_mfpt(o, succ, absorbing)
    np.testing.assert_allclose(tg, to, rtol=1e-10, atol=0)
