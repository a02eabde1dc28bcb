"""Host logic of the serving loop on the CPU: admission order (FIFO, or
largest expected work first with the Eq. 10 workload proxy), the expected
work of event and time horizons, request validation, shape classes and the
latency summary."""
import types

import numpy as np
import pytest

import synth
from paper_2604_24091_gb300 import serve


def _req(t, T, rid, n=0, t_sim=0.0, L=32, nv=1, model=synth.EAM_MODEL):
    d = synth.VoxelDesc(L, nv, (0.003, 0.007, 0.014), T, model, synth.PREC_SPLIT, seed=rid, uid=rid)
    return serve.Request(t, d, n_events=n, rid=rid, t_sim=t_sim)


def _srv(policy):
    return types.SimpleNamespace(policy=policy, nu=6e12)


def test_fifo_admission_is_arrival_order():
    srv = _srv("fifo")
    reqs = [_req(t, 563.0, i, n=1000) for i, t in enumerate([0.3, 0.1, 0.2, 0.1])]
    order = sorted(reqs, key=lambda r: serve.Server._priority(srv, r, 1.0))
    assert [r.rid for r in order] == [1, 3, 2, 0]


def test_proxy_orders_by_expected_work():
    srv = _srv("proxy")
    # W0 per request (Gamma_tot / nu of its initial state): a time horizon's work
    # is nu W0 t_sim, an event horizon's its event count
    w0 = {0: 2e-5, 1: 8e-5, 2: 4e-5}
    reqs = [_req(0.0, 563.0, 0, t_sim=1e-3), _req(0.1, 563.0, 1, t_sim=1e-3), _req(0.2, 563.0, 2, t_sim=3e-3),
            _req(0.3, 563.0, 3, n=700000), _req(0.4, 563.0, 4, n=100)]
    work = {r.rid: serve.Server._expected_work(srv, r, w0) for r in reqs}
    assert work == pytest.approx({0: 6e12 * 2e-5 * 1e-3, 1: 6e12 * 8e-5 * 1e-3, 2: 6e12 * 4e-5 * 3e-3,
                                  3: 700000.0, 4: 100.0}, rel=1e-15)
    order = [r.rid for r in sorted(reqs, key=lambda r: serve.Server._priority(srv, r, work[r.rid]))]
    assert order == [2, 3, 1, 0, 4]
    # equal work falls back to arrival order
    twins = [_req(0.5, 563.0, 7, n=1000), _req(0.2, 563.0, 8, n=1000)]
    assert [r.rid for r in sorted(twins, key=lambda r: serve.Server._priority(srv, r, 1000.0))] == [8, 7]


def test_shape_class_ignores_temperature_composition_precision():
    a = _req(0.0, 543.0, 1, n=1)
    b = _req(0.0, 593.0, 2, n=1)
    b.desc.precision = synth.PREC_FP64
    assert serve.shape_class(a.desc) == serve.shape_class(b.desc) == (32, 1, synth.EAM_MODEL)
    assert serve.shape_class(_req(0, 563.0, 3, n=1, L=16).desc) != serve.shape_class(a.desc)
    assert serve.shape_class(_req(0, 563.0, 3, n=1, model=synth.PAIR_MODEL).desc) != serve.shape_class(a.desc)


def test_policy_and_horizon_validation():
    with pytest.raises(ValueError):
        serve.Server(synth.default_model(), policy="lifo")


def test_latency_summary_percentiles():
    res = [serve.Result(i, arrival=0.0, admitted=0.0, finished=float(i + 1), n_events=int(2e6), status=0)
           for i in range(100)]
    s = serve.latency_summary(res)
    lat = np.arange(1, 101, dtype=np.float64)
    assert s["requests"] == 100
    assert s["p50_latency_s"] == np.percentile(lat, 50)
    assert s["p99_s_per_1e6"] == np.percentile(lat / 2.0, 99)
    assert s["makespan_s"] == 100.0
    assert serve.latency_summary([]) == {}
