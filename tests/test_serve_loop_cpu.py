"""The serving loop on the CPU with a stand-in batch (no GPU): every request
finishes, each once; requests of several shape classes share one HBM budget;
a budget that cannot hold a class raises instead of waiting forever; time
horizons are met; proxy admission follows the expected work.  The stand-in
only counts events and advances a clock at a fixed rate per voxel (Gamma =
nu W, W from the temperature), which is all the loop reads."""
import math

import numpy as np
import pytest

import synth
from paper_2604_24091_gb300 import serve

NU = 6e12
SLOT = 1000          # bytes per slot of the stand-in (any class)
BASE = 500


def _w(desc):
    return 8 * desc.n_vac * math.exp(-0.62 / (8.617333262e-5 * desc.T))


class FakeBatch:
    live = 0

    def __init__(self, descs, model, **kw):
        self.descs = list(descs)
        self.n = len(self.descs)
        self.nbytes = BASE + SLOT * self.n
        self.ev = np.zeros(self.n, np.int64)
        self.t = np.zeros(self.n)
        FakeBatch.live += 1

    def close(self):
        FakeBatch.live -= 1

    def set_launch(self, *a):
        pass

    def reset_voxels(self, slots, descs, stream=None):
        for s, d in zip(slots, descs):
            assert serve.shape_class(d) == serve.shape_class(self.descs[s])
            self.descs[s] = d
            self.ev[s] = 0
            self.t[s] = 0.0

    def step(self, n, stream=None):
        n = np.asarray(n, np.int64)
        for s in range(self.n):
            self.ev[s] += n[s]
            self.t[s] += n[s] / (NU * _w(self.descs[s]))

    def workload_proxy(self, stream=None):
        W = np.array([_w(d) for d in self.descs])
        M = np.array([8.0 * d.n_vac for d in self.descs])
        return W, M, np.full(self.n, 0.62)

    def read_batch_state(self, out, stream=None):
        out["t_hi"][:] = self.t
        out["t_lo"][:] = 0.0

    def sync_status(self, stream=None):
        return 0, np.zeros(self.n, np.int32)

    def read_state(self, v, stream=None):
        return {"n_events": int(self.ev[v]), "t_hi": float(self.t[v]), "t_lo": 0.0}


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    monkeypatch.setattr(serve, "workspace_bytes", lambda descs, model, *a: BASE + SLOT * len(descs))
    FakeBatch.live = 0
    return FakeBatch


def _req(rid, L, nv, T, n=0, t_sim=0.0, model=synth.EAM_MODEL, t=0.0):
    d = synth.VoxelDesc(L, nv, (0.01, 0.01, 0.01), T, model, synth.PREC_SPLIT, seed=rid + 1, uid=rid)
    return serve.Request(t, d, n_events=n, rid=rid, t_sim=t_sim)


def test_mixed_classes_all_finish_under_budget(fake):
    rng = np.random.default_rng(1)
    reqs = []
    for i in range(60):
        L = int(rng.choice([16, 24, 32]))
        nv = int(rng.integers(1, 3))
        if i % 2:
            reqs.append(_req(i, L, nv, float(rng.uniform(543, 593)), n=int(rng.integers(1000, 90000))))
        else:
            reqs.append(_req(i, L, nv, float(rng.uniform(543, 593)), t_sim=float(rng.uniform(1e-4, 1e-3))))
    srv = serve.Server(synth.default_model(), hbm_budget=BASE * 12 + SLOT * 40, chunk=20000, min_pool=2, max_pool=8)
    res, st = srv.run(reqs, collect_state=True, realtime=False)
    assert sorted(r.rid for r in res) == list(range(60))
    assert srv.used_bytes <= BASE * 12 + SLOT * 40
    for r in res:
        q = reqs[r.rid]
        if q.n_events:
            assert r.n_events == r.state["n_events"] == q.n_events
        else:
            assert r.t_sim >= q.t_sim
            # the last round ran at most 0.9 Gamma dt_left + 1 events: overshoot below 2 events
            assert r.t_sim - q.t_sim < 2.0 / (NU * _w(q.desc))
    srv.close()
    assert fake.live == 0


def test_budget_too_small_for_a_class_raises(fake):
    srv = serve.Server(synth.default_model(), hbm_budget=BASE + SLOT - 1, chunk=1000)
    with pytest.raises(RuntimeError, match="cannot hold a slot"):
        srv.run([_req(0, 16, 1, 563.0, n=10)], realtime=False)


def test_idle_pools_are_released_for_another_class(fake):
    # room for one pool of 4 slots at a time: the classes take turns
    srv = serve.Server(synth.default_model(), hbm_budget=BASE + 4 * SLOT, chunk=1000, min_pool=4, max_pool=4)
    reqs = [_req(i, 16 if i < 6 else 24, 1, 563.0, n=3000) for i in range(12)]
    res, st = srv.run(reqs, realtime=False)
    assert len(res) == 12 and all(r.n_events == 3000 for r in res)
    assert st["pools"] == 1


def test_proxy_admits_largest_expected_work_first(fake):
    # one slot: admissions happen one by one, in the order of nu W0 t_sim (time
    # horizons, W0 of the initial state) or n_events (event horizons)
    reqs = [_req(0, 16, 1, 550.0, t_sim=1e-4), _req(1, 16, 1, 590.0, t_sim=1e-4), _req(2, 16, 1, 570.0, n=5000),
            _req(3, 16, 1, 590.0, t_sim=3e-4), _req(4, 16, 1, 545.0, n=100)]
    work = {r.rid: (r.n_events if r.n_events else NU * _w(r.desc) * r.t_sim) for r in reqs}
    srv = serve.Server(synth.default_model(), hbm_budget=BASE + 1.5 * SLOT, chunk=10 ** 6, policy="proxy",
                       min_pool=1, max_pool=1)
    res, _ = srv.run(reqs, realtime=False)
    assert [r.rid for r in sorted(res, key=lambda r: r.admitted)] == sorted(work, key=lambda k: -work[k])
    for r in res:
        assert r.expected_work == pytest.approx(work[r.rid], rel=1e-12)
