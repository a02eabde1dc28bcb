"""Continuous batching of voxel AKMC requests on one GPU.

A request is one voxel simulation (a descriptor and a number of events).  The
server keeps a fixed pool of voxel slots resident in one workspace (sized by
an HBM budget), admits arrived requests into free slots as they free up
(akmc_reset_voxels re-seeds a slot in place), and advances every occupied
slot by at most `chunk` events per persistent launch.  Requests that arrive
while others run join at the next launch boundary; their work overlaps on the
device with the requests already running.  Each request's result is the same
as running it alone: its random stream depends only on (seed, uid, event
index) and its arithmetic only on its own voxel.

Admission order is FIFO, or largest workload proxy first (W ~ M exp(-E/kT)
with M the requested events and E the Fe migration barrier; the paper's
dynamic voxel scheduling, Eq. 10).
"""
from __future__ import annotations

import collections
import dataclasses
import heapq
import math
import time
from typing import List, Optional, Sequence

import numpy as np

from .akmc import Batch, workspace_bytes

KB_EV = 8.617333262e-5


@dataclasses.dataclass
class Request:
    arrival: float          # seconds from the start of the run
    desc: object            # voxel descriptor (same L, n_vac, model, precision as the slots)
    n_events: int
    rid: int = 0


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    n_events: int
    status: int
    state: Optional[dict] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def latency_per_1e6(self) -> float:
        return self.latency / (self.n_events / 1e6)


class Server:
    def __init__(self, model, shape, n_slots: Optional[int] = None, hbm_budget: float = 120e9,
                 chunk: int = 50000, max_slots: int = 4096, policy: str = "fifo", launch=None):
        """`shape`: a descriptor whose L, n_vac, model and precision every request shares."""
        self.shape = shape
        self.model = model
        one = workspace_bytes([shape], model)
        two = workspace_bytes([shape, shape], model)
        per_slot = max(1, two - one)
        fit = int((hbm_budget - one) // per_slot) + 1
        self.n_slots = min(max_slots, fit) if n_slots is None else min(n_slots, fit)
        if self.n_slots < 1:
            raise ValueError("HBM budget %.3g B holds no voxel of this shape" % hbm_budget)
        self.bytes_per_slot = per_slot
        idle = [dataclasses.replace(shape, uid=(1 << 62) + s, seed=s + 1) for s in range(self.n_slots)]
        self.batch = Batch(idle, model)
        if launch is not None:
            self.batch.set_launch(*launch)
        self.chunk = int(chunk)
        self.policy = policy

    def _priority(self, req: Request):
        if self.policy == "proxy":
            w = req.n_events * math.exp(-self.model.E0[0] / (KB_EV * req.desc.T))
            return (-w, req.arrival, req.rid)
        return (req.arrival, req.rid)

    def run(self, requests: Sequence[Request], collect_state: bool = False, realtime: bool = True):
        """Serve `requests` (arrival times relative to the start).  With
        realtime=False arrivals are taken as already due (offline batch)."""
        import torch
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        pending = collections.deque(reqs)
        waiting: List = []
        free = list(range(self.n_slots - 1, -1, -1))
        active = {}                        # slot -> [request, remaining, admitted]
        results: List[Result] = []
        targets = np.zeros(self.n_slots, np.uint64)
        total_events = 0
        t0 = time.perf_counter()
        now = lambda: (time.perf_counter() - t0) if realtime else float("inf")
        busy = 0.0
        launches = 0
        while pending or waiting or active:
            tnow = now()
            while pending and pending[0].arrival <= tnow:
                r = pending.popleft()
                heapq.heappush(waiting, (self._priority(r), r.rid, r))
            slots, descs = [], []
            while free and waiting:
                r = heapq.heappop(waiting)[2]
                s = free.pop()
                slots.append(s)
                descs.append(r.desc)
                active[s] = [r, int(r.n_events), min(tnow, time.perf_counter() - t0)]
            if slots:
                self.batch.reset_voxels(slots, descs)
            if not active:
                if pending:
                    wait = pending[0].arrival - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                continue
            targets[:] = 0
            for s, (r, rem, _) in active.items():
                targets[s] = min(rem, self.chunk)
            tl = time.perf_counter()
            self.batch.step(targets)
            torch.cuda.current_stream().synchronize()
            busy += time.perf_counter() - tl
            launches += 1
            tdone = time.perf_counter() - t0
            total_events += int(targets.sum())
            done = []
            for s, entry in active.items():
                entry[1] -= int(targets[s])
                if entry[1] <= 0:
                    done.append(s)
            if done:
                _, per = self.batch.sync_status()
                for s in done:
                    r, _, adm = active.pop(s)
                    st = self.batch.read_state(s) if collect_state else None
                    results.append(Result(r.rid, r.arrival, adm, tdone, int(r.n_events), int(per[s]), st))
                    free.append(s)
        elapsed = time.perf_counter() - t0
        return results, {"elapsed_s": elapsed, "busy_s": busy, "events": total_events, "launches": launches,
                         "events_per_s": total_events / max(elapsed, 1e-9), "slots": self.n_slots,
                         "bytes_per_slot": self.bytes_per_slot}


def latency_summary(results: Sequence[Result]):
    lat = np.array([r.latency_per_1e6 for r in results])
    if lat.size == 0:
        return {}
    return {"requests": int(lat.size), "p50_s_per_1e6": float(np.percentile(lat, 50)),
            "p99_s_per_1e6": float(np.percentile(lat, 99)),
            "p50_latency_s": float(np.percentile([r.latency for r in results], 50)),
            "p99_latency_s": float(np.percentile([r.latency for r in results], 99))}
