"""GPU: CUDA-graph replay of the step, in-place slot re-seeding, and the
continuous-batching server (each result equal to the same request run alone)."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from oracle.proxy import workload_proxy

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2604_24091_gb300 import Batch, workspace_bytes  # noqa: E402
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


def _mixed_requests(rng, n, t0=0.0, dt=0.002):
    """Requests of different sizes, vacancy counts, models, precisions,
    compositions and temperatures; event or simulated-time horizons."""
    shapes = [(6, 1, synth.PAIR_MODEL, synth.PREC_FP64), (8, 1, synth.EAM_MODEL, synth.PREC_SPLIT),
              (8, 1, synth.EAM_MODEL, synth.PREC_FP64), (7, 3, synth.EAM_MODEL, synth.PREC_SPLIT),
              (10, 2, synth.PAIR_MODEL, synth.PREC_FP64)]
    reqs = []
    for i in range(n):
        L, nv, mdl, prec = shapes[i % len(shapes)]
        d = synth.VoxelDesc(L, nv, tuple(float(x) for x in rng.uniform(0.01, 0.05, 3)), float(rng.uniform(543, 593)),
                            mdl, prec, seed=int(rng.integers(1, 1 << 62)), uid=1000 + i)
        if i % 3 == 2:
            reqs.append(Request(arrival=t0 + dt * i, desc=d, t_sim=float(rng.uniform(2e-5, 8e-5)), rid=i))
        else:
            reqs.append(Request(arrival=t0 + dt * i, desc=d, n_events=int(rng.integers(1000, 6000)), rid=i))
    return reqs


def _same_state(m, s):
    assert m["n_events"] == s["n_events"]
    assert np.array_equal(m["species"], s["species"])
    assert np.array_equal(m["vac_disp"], s["vac_disp"])
    t_m, t_s = m["t_hi"] + m["t_lo"], s["t_hi"] + s["t_lo"]
    assert abs(t_m - t_s) <= 1e-12 * t_s


def test_server_mixed_shapes_equal_alone(model):
    rng = np.random.default_rng(4)
    reqs = _mixed_requests(rng, 15)
    srv = Server(model, hbm_budget=64e6, chunk=1700, min_pool=2)
    results, stats = srv.run(reqs, collect_state=True)
    assert len(results) == len(reqs)
    assert all(r.status == 0 for r in results)
    assert stats["pools"] >= 4                      # one shape class per pool at least
    by_id = {r.rid: r for r in results}
    for q in reqs:
        res = by_id[q.rid]
        if q.n_events:
            alone = Batch([q.desc], model)
            alone.step(q.n_events)
            s = alone.read_state(0)
            assert res.n_events == q.n_events
        else:
            # a time horizon: the rounds' targets depend on the voxel's own state only
            solo = Server(model, hbm_budget=8e6, chunk=1700, min_pool=1)
            (r1,), _ = solo.run([Request(0.0, q.desc, t_sim=q.t_sim, rid=q.rid)], collect_state=True)
            solo.close()
            s = r1.state
            assert res.t_sim >= q.t_sim and res.n_events == r1.n_events
        _same_state(res.state, s)
    srv.close()
    summ = latency_summary(results)
    assert summ["p99_s_per_1e6"] >= summ["p50_s_per_1e6"] > 0


def test_time_horizon_stops_at_first_round_past_t_sim(model):
    d = synth.VoxelDesc(8, 1, (0.02, 0.02, 0.02), 563.0, synth.EAM_MODEL, synth.PREC_SPLIT, seed=9, uid=9)
    srv = Server(model, hbm_budget=8e6, chunk=100000, min_pool=1)
    (r,), _ = srv.run([Request(0.0, d, t_sim=3e-4, rid=0)], collect_state=True)
    srv.close()
    t = r.state["t_hi"] + r.state["t_lo"]
    assert t >= 3e-4
    # the last round asked for at most 0.9 Gamma_tot dt_left + 1 events: the clock
    # overshoots by a few mean residence times at most
    b = Batch([d], model)
    W, _, _ = b.workload_proxy()
    mean_dt = 1.0 / (model.nu * W[0])
    assert t - 3e-4 < 40 * mean_dt
    assert r.n_events == r.state["n_events"]


def test_proxy_admission_order_follows_initial_state_work(model):
    # slots for one request at a time: the proxy policy admits the largest
    # nu W0 t_sim first, W0 the workload proxy of the request's initial state
    # (computed here by the oracle)
    rng = np.random.default_rng(11)
    reqs = []
    for i, T in enumerate((545.0, 590.0, 560.0, 575.0, 550.0)):
        d = synth.VoxelDesc(8, 1, (0.02, 0.01, 0.01), T, synth.EAM_MODEL, synth.PREC_SPLIT,
                            seed=int(rng.integers(1, 1 << 40)), uid=200 + i)
        reqs.append(Request(0.0, d, t_sim=2e-5, rid=i))
    # room for one single-slot pool (or a one-slot probe batch): one request at a time
    budget = 1.5 * workspace_bytes([reqs[0].desc], model)
    srv = Server(model, hbm_budget=budget, chunk=400000, policy="proxy", min_pool=1, max_pool=1)
    results, _ = srv.run(reqs, realtime=False)
    srv.close()
    work = {}
    for q in reqs:
        o = oracle.Voxel(q.desc, model)
        W0, _, _ = workload_proxy(o.state()["rates"], q.desc.T, model.nu)
        work[q.rid] = model.nu * W0 * q.t_sim
    for r in results:
        # split-precision rates: within beta x 1e-5 eV (relative) of the float64 oracle
        assert abs(r.expected_work - work[r.rid]) <= 2.2e-4 * work[r.rid]
    order = [r.rid for r in sorted(results, key=lambda r: r.admitted)]
    assert order == sorted(work, key=lambda k: -work[k])


def test_server_slots_follow_the_hbm_budget(model):
    proto = synth.VoxelDesc(32, 1, (0.003, 0.007, 0.014), 563.0, synth.EAM_MODEL, synth.PREC_SPLIT)
    srv = Server(model, hbm_budget=40e6, reserve=[(proto, 10000)])
    assert srv.used_bytes <= 40e6
    assert 50 <= srv.n_slots <= 130
    srv.close()
