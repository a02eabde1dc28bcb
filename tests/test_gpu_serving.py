"""GPU: CUDA-graph replay of the step, in-place slot re-seeding, and the
continuous-batching server (each result equal to the same request run alone)."""
import dataclasses

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2604_24091_gb300 import Batch  # noqa: E402
from paper_2604_24091_gb300.serve import Request, Server, latency_summary  # noqa: E402


def _descs():
    return [synth.VoxelDesc(6, 2, (0.05, 0.05, 0.05), 563.0, synth.PAIR_MODEL, synth.PREC_FP64, seed=5, uid=50),
            synth.VoxelDesc(8, 1, (0.04, 0.04, 0.04), 553.0, synth.EAM_MODEL, synth.PREC_SPLIT, seed=6, uid=51),
            synth.VoxelDesc(7, 3, (0.06, 0.02, 0.02), 583.0, synth.EAM_MODEL, synth.PREC_FP64, seed=7, uid=52)]


def test_graph_replay_equals_step(model):
    descs = _descs()
    a = Batch(descs, model, event_log_capacity=2000)
    b = Batch(descs, model, event_log_capacity=2000)
    for _ in range(4):
        a.step(500)
    g = b.capture_step(500)
    for _ in range(4):
        g.replay()
    torch.cuda.synchronize()
    for v in range(len(descs)):
        sa, sb = a.read_state(v, log=True), b.read_state(v, log=True)
        assert sa["n_events"] == sb["n_events"] == 2000
        assert np.array_equal(sa["event_log"], sb["event_log"])
        assert np.array_equal(sa["species"], sb["species"])
        assert sa["t_hi"] == sb["t_hi"] and sa["t_lo"] == sb["t_lo"]


def test_reset_voxel_equals_fresh_voxel(model):
    descs = _descs()
    b = Batch(descs, model, event_log_capacity=1500)
    b.step(700)
    new = dataclasses.replace(descs[1], T=591.0, frac=(0.02, 0.06, 0.03), seed=99, uid=77)
    b.reset_voxels([1], [new])
    b.step(1500)
    f = Batch([new], model, event_log_capacity=1500)
    f.step(1500)
    g1, g2 = b.read_state(1, log=True), f.read_state(0, log=True)
    assert g1["n_events"] == g2["n_events"] == 1500
    assert np.array_equal(g1["event_log"], g2["event_log"])
    assert np.array_equal(g1["species"], g2["species"])
    assert g1["t_hi"] == g2["t_hi"] and g1["t_lo"] == g2["t_lo"]
    # the other voxels were not disturbed
    c = Batch(descs, model)
    c.step(2200)
    for v in (0, 2):
        assert np.array_equal(b.read_state(v)["species"], c.read_state(v)["species"])


def test_server_results_equal_alone(model):
    shape = synth.VoxelDesc(8, 1, (0.03, 0.03, 0.03), 563.0, synth.EAM_MODEL, synth.PREC_SPLIT)
    rng = np.random.default_rng(4)
    reqs = []
    for i in range(14):
        d = dataclasses.replace(shape, T=float(rng.uniform(543, 593)),
                                frac=tuple(float(x) for x in rng.uniform(0.01, 0.05, 3)),
                                seed=int(rng.integers(1, 1 << 62)), uid=1000 + i)
        reqs.append(Request(arrival=0.002 * i, desc=d, n_events=int(rng.integers(1000, 6000)), rid=i))
    srv = Server(model, shape, n_slots=5, chunk=1700)
    results, stats = srv.run(reqs, collect_state=True)
    assert len(results) == len(reqs) and stats["events"] == sum(r.n_events for r in reqs)
    assert all(r.status == 0 for r in results)
    by_id = {r.rid: r for r in results}
    for q in reqs:
        alone = Batch([q.desc], model)
        alone.step(q.n_events)
        s = alone.read_state(0)
        m = by_id[q.rid].state
        assert m["n_events"] == s["n_events"] == q.n_events
        assert np.array_equal(m["species"], s["species"])
        assert np.array_equal(m["vac_disp"], s["vac_disp"])
        t_m, t_s = m["t_hi"] + m["t_lo"], s["t_hi"] + s["t_lo"]
        assert abs(t_m - t_s) <= 1e-12 * t_s
    summ = latency_summary(results)
    assert summ["p99_s_per_1e6"] >= summ["p50_s_per_1e6"] > 0


def test_server_slots_follow_the_hbm_budget(model):
    shape = synth.VoxelDesc(32, 1, (0.003, 0.007, 0.014), 563.0, synth.EAM_MODEL, synth.PREC_SPLIT)
    srv = Server(model, shape, hbm_budget=40e6)
    assert srv.n_slots * srv.bytes_per_slot <= 40e6 + srv.bytes_per_slot
    assert 50 <= srv.n_slots <= 130
