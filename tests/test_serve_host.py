"""Host logic of the serving loop on the CPU: admission order (FIFO, or the
workload proxy W ~ M exp(-E/kT) of the paper's dynamic voxel scheduling,
Eq. 10, largest first) and the latency summary."""
import math
import types

import numpy as np

import synth
from paper_2604_24091_gb300 import serve


def _req(t, T, n, rid):
    d = synth.VoxelDesc(32, 1, (0.003, 0.007, 0.014), T, synth.EAM_MODEL, synth.PREC_SPLIT, seed=rid, uid=rid)
    return serve.Request(t, d, n, rid)


def test_proxy_admission_is_largest_expected_work_first():
    model = synth.default_model()
    srv = types.SimpleNamespace(policy="proxy", model=model)
    reqs = [_req(0.1 * i, T, n, i) for i, (T, n) in enumerate(
        [(543.0, 5e6), (593.0, 1e6), (563.0, 2e6), (593.0, 4e6), (543.0, 1e7)])]
    order = sorted(reqs, key=lambda r: serve.Server._priority(srv, r))
    W = [r.n_events * math.exp(-model.E0[0] / (serve.KB_EV * r.desc.T)) for r in order]
    assert all(W[i] >= W[i + 1] for i in range(len(W) - 1))
    # ties in W fall back to arrival order
    twins = [_req(0.5, 563.0, 1e6, 7), _req(0.2, 563.0, 1e6, 8)]
    assert [r.rid for r in sorted(twins, key=lambda r: serve.Server._priority(srv, r))] == [8, 7]


def test_fifo_admission_is_arrival_order():
    srv = types.SimpleNamespace(policy="fifo", model=synth.default_model())
    reqs = [_req(t, 563.0, 1e6, i) for i, t in enumerate([0.3, 0.1, 0.2, 0.1])]
    order = sorted(reqs, key=lambda r: serve.Server._priority(srv, r))
    assert [r.rid for r in order] == [1, 3, 2, 0]


def test_latency_summary_percentiles():
    res = [serve.Result(i, arrival=0.0, admitted=0.0, finished=float(i + 1), n_events=int(2e6), status=0)
           for i in range(100)]
    s = serve.latency_summary(res)
    lat = np.arange(1, 101, dtype=np.float64)
    assert s["requests"] == 100
    assert s["p50_latency_s"] == np.percentile(lat, 50)
    assert s["p99_s_per_1e6"] == np.percentile(lat / 2.0, 99)
    assert serve.latency_summary([]) == {}
