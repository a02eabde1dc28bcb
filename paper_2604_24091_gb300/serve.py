"""Continuous batching of voxel AKMC requests on one GPU.

A request is one voxel simulation: a descriptor plus a horizon, either a
number of events or a span of simulated time.  Voxels of any size,
composition, temperature, model and precision are served side by side.

Memory.  Slots live in pools; a pool is one batch (one workspace) of slots
that share a shape class (edge L, vacancy count, energy model).  Pools are
created on demand under one HBM budget -- the first pool of a class holds
`min_pool` slots and each further one twice as many as the last, up to
`max_pool` -- and a pool with no active slot is released when another class
needs its memory.  A request waits until a slot of its class is free or the
budget allows a new pool.  A slot takes a new request in place
(akmc_reset_voxels: fresh placement, densities, rates and tree; the
precision may change).

Compute.  Every round, each pool with active slots runs one persistent
launch on its own CUDA stream, so the pools' work overlaps on the device;
a slot advances by at most `chunk` events per round.  Requests that arrive
while others run are admitted at the next round.  A request's result equals
running it alone: its random stream depends only on (seed, uid, event
index), its arithmetic only on its own voxel, and the targets of its rounds
only on its own state.

Scheduling (the paper's dynamic voxel scheduling, Sec. "Dynamic Voxel
Scheduling", Eq. 10).  The workload proxy W = M_hat exp(-E_hat / kT) of a
voxel comes from its current state on the device (akmc_workload_proxy):
M_hat the number of admissible hops, E_hat the effective barrier that gives
each of them the voxel's mean rate, so nu W is the voxel's event rate and a
span dt of simulated time takes about nu W dt events.  With policy "proxy"
waiting requests are admitted largest expected work first (events for an
event horizon; nu W0 t_sim for a time horizon, W0 from the request's initial
state, evaluated in a small probe batch of its class); with "fifo" in
arrival order.  A time-horizon request runs in rounds of at most
0.9 nu W dt_left + 1 events (re-estimated from its live state each round)
until its clock reaches t_sim; it ends at the end of that round.
Inside each launch the persistent kernel's work queue hands out the voxels
with the most work first.
"""
from __future__ import annotations

import collections
import dataclasses
import heapq
import math
import time
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from .akmc import Batch, workspace_bytes

NU_DEFAULT = 6.0e12


@dataclasses.dataclass
class Request:
    arrival: float          # seconds from the start of the run
    desc: object            # voxel descriptor
    n_events: int = 0       # events to run (event horizon), or 0 with t_sim > 0
    rid: int = 0
    t_sim: float = 0.0      # simulated seconds to advance (time horizon)


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    n_events: int           # events run
    status: int
    state: Optional[dict] = None
    t_sim: float = 0.0      # simulated time reached (time-horizon requests)
    expected_work: float = 0.0

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def latency_per_1e6(self) -> float:
        return self.latency / (max(self.n_events, 1) / 1e6)


def shape_class(desc) -> Tuple[int, int, int]:
    return (int(desc.L), int(desc.n_vac), int(desc.model))


class _Pool:
    def __init__(self, key, proto, n_slots, model, launch, uid0):
        import torch
        self.key = key
        idle = [dataclasses.replace(proto, uid=uid0 + s, seed=uid0 + s + 1) for s in range(n_slots)]
        self.nbytes = workspace_bytes(idle, model)
        self.batch = Batch(idle, model)
        if launch is not None:
            self.batch.set_launch(*launch)
        self.n = n_slots
        self.free = list(range(n_slots - 1, -1, -1))
        self.active: Dict[int, list] = {}
        self.stream = torch.cuda.Stream() if torch.cuda.is_available() else None

    def close(self):
        self.batch.close()
        self.batch = None


class Server:
    def __init__(self, model, hbm_budget: float = 120e9, chunk: int = 50000, policy: str = "fifo",
                 min_pool: int = 16, max_pool: int = 2048, reserve: Sequence = (), launch=None,
                 probe_slots: int = 16):
        """`reserve`: (prototype descriptor, slots) pairs, pools created up front
        (each descriptor stands for its shape class)."""
        if policy not in ("fifo", "proxy"):
            raise ValueError("policy must be 'fifo' or 'proxy'")
        self.model = model
        self.budget = float(hbm_budget)
        self.chunk = int(chunk)
        self.policy = policy
        self.min_pool, self.max_pool = int(min_pool), int(max_pool)
        self.launch = launch
        self.probe_slots = int(probe_slots)
        self.nu = float(getattr(model, "nu", NU_DEFAULT))
        self.pools: List[_Pool] = []
        self._uid = 1 << 62
        self._grow: Dict[Tuple, int] = collections.defaultdict(int)
        for proto, k in reserve:
            if self._new_pool(proto, int(k)) is None:
                raise ValueError("HBM budget %.3g B holds no pool of %d slots of class %s"
                                 % (self.budget, k, shape_class(proto)))

    # -------------------------------------------------------------- memory
    @property
    def used_bytes(self) -> int:
        return sum(p.nbytes for p in self.pools)

    @property
    def n_slots(self) -> int:
        return sum(p.n for p in self.pools)

    def slot_bytes(self, proto) -> int:
        one = workspace_bytes([proto], self.model)
        two = workspace_bytes([proto, proto], self.model)
        return max(1, two - one)

    def _new_pool(self, proto, k):
        key = shape_class(proto)
        base = workspace_bytes([proto], self.model) - self.slot_bytes(proto)
        per = self.slot_bytes(proto)
        room = self.budget - self.used_bytes
        if room < base + per:
            # release idle pools of other classes, largest first
            idle = sorted((p for p in self.pools if not p.active and p.key != key), key=lambda p: -p.nbytes)
            for p in idle:
                if room >= base + per * k:
                    break
                self.pools.remove(p)
                p.close()
                room = self.budget - self.used_bytes
        k = int(min(k, (room - base) // per))
        if k < 1:
            return None
        pool = _Pool(key, proto, k, self.model, self.launch, self._uid)
        self._uid += k
        self.pools.append(pool)
        return pool

    def _slot_for(self, desc):
        key = shape_class(desc)
        for p in self.pools:
            if p.key == key and p.free:
                return p
        g = self._grow[key]
        want = min(self.max_pool, self.min_pool << g)
        pool = self._new_pool(desc, want)
        if pool is not None:
            self._grow[key] = g + 1
        return pool

    # --------------------------------------------------------- scheduling
    def _probe_w0(self, reqs):
        """W0 = Gamma_tot / nu of each time-horizon request's initial state, from
        a transient probe batch of its shape class (placement and rates only),
        sized within the free part of the HBM budget and released after use."""
        by_key = collections.defaultdict(list)
        for r in reqs:
            by_key[shape_class(r.desc)].append(r)
        out = {}
        for key, rs in by_key.items():
            per = self.slot_bytes(rs[0].desc)
            base = workspace_bytes([rs[0].desc], self.model) - per
            k = int(min(self.probe_slots, len(rs), (self.budget - self.used_bytes - base) // per))
            if k < 1:
                continue                # no room to probe now: the request keeps work 0 (admitted last)
            pb = _Pool(key, rs[0].desc, k, self.model, None, self._uid)
            self._uid += k
            for i in range(0, len(rs), k):
                part = rs[i:i + k]
                pb.batch.reset_voxels(list(range(len(part))), [r.desc for r in part])
                W, _, _ = pb.batch.workload_proxy()
                for j, r in enumerate(part):
                    out[r.rid] = float(W[j])
            pb.close()
        return out

    def _expected_work(self, r, w0):
        if r.n_events > 0:
            return float(r.n_events)
        return self.nu * w0.get(r.rid, 0.0) * float(r.t_sim)

    def _priority(self, r, work):
        if self.policy == "proxy":
            return (-work, r.arrival, r.rid)
        return (r.arrival, r.rid)

    # ---------------------------------------------------------------- run
    def run(self, requests: Sequence[Request], collect_state: bool = False, realtime: bool = True):
        """Serve `requests` (arrival times relative to the start).  With
        realtime=False arrivals are taken as already due (offline batch)."""
        import torch
        for r in requests:
            if not ((r.n_events > 0) ^ (r.t_sim > 0)):
                raise ValueError("request %d: give n_events or t_sim" % r.rid)
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        pending = collections.deque(reqs)
        waiting: List = []
        results: List[Result] = []
        total_events = 0
        t0 = time.perf_counter()
        now = lambda: (time.perf_counter() - t0) if realtime else float("inf")
        busy = 0.0
        launches = 0
        w0: Dict[int, float] = {}
        while pending or waiting or any(p.active for p in self.pools):
            tnow = now()
            arrived = []
            while pending and pending[0].arrival <= tnow:
                arrived.append(pending.popleft())
            if arrived and self.policy == "proxy":
                w0.update(self._probe_w0([r for r in arrived if r.t_sim > 0]))
            for r in arrived:
                work = self._expected_work(r, w0)
                heapq.heappush(waiting, (self._priority(r, work), r.rid, r, work))
            # admission: in priority order, while a slot of the class is free or
            # the budget allows a new pool
            blocked, resets = [], collections.defaultdict(list)
            tadm = min(tnow, time.perf_counter() - t0)
            while waiting:
                item = heapq.heappop(waiting)
                r = item[2]
                pool = self._slot_for(r.desc)
                if pool is None:
                    blocked.append(item)
                    continue
                s = pool.free.pop()
                pool.active[s] = [r, int(r.n_events), tadm, 0, item[3]]   # request, events left, admitted, run, work
                resets[id(pool)].append((pool, s, r.desc))
            for item in blocked:
                heapq.heappush(waiting, item)
            for lst in resets.values():
                pool = lst[0][0]
                pool.batch.reset_voxels([s for _, s, _ in lst], [d for _, _, d in lst], stream=pool.stream)
            live = [p for p in self.pools if p.active]
            if not live and waiting and not pending:
                # nothing runs, nothing more arrives, and the waiting requests found no room
                raise RuntimeError("HBM budget %.3g B cannot hold a slot for request %d (class %s)"
                                   % (self.budget, waiting[0][2].rid, shape_class(waiting[0][2].desc)))
            if not live:
                if pending:
                    wait = pending[0].arrival - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                continue
            # targets of this round
            tl = time.perf_counter()
            plans = []
            for p in live:
                tg = np.zeros(p.n, np.uint64)
                stalled = set()
                if any(e[0].t_sim > 0 for e in p.active.values()):
                    W, _, _ = p.batch.workload_proxy(stream=p.stream)
                    clk = self._clocks(p)
                for s, e in p.active.items():
                    r = e[0]
                    if r.t_sim > 0:
                        if not (W[s] > 0.0 and math.isfinite(W[s])):
                            stalled.add(s)      # no admissible event (or a numeric error): the clock cannot move
                            continue
                        left = r.t_sim - clk[s]
                        tg[s] = min(self.chunk, int(0.9 * self.nu * W[s] * left) + 1)
                    else:
                        tg[s] = min(e[1], self.chunk)
                p.batch.step(tg, stream=p.stream)
                plans.append((p, tg, stalled))
            for p, _, _ in plans:
                if p.stream is not None:
                    p.stream.synchronize()
            busy += time.perf_counter() - tl
            launches += 1
            tdone = time.perf_counter() - t0
            for p, tg, stalled in plans:
                total_events += int(tg.sum())
                done = []
                timed = any(e[0].t_sim > 0 for e in p.active.values())
                clk = self._clocks(p) if timed else None
                for s, e in p.active.items():
                    e[3] += int(tg[s])
                    if e[0].t_sim > 0:
                        if s in stalled or clk[s] >= e[0].t_sim:
                            done.append(s)
                    else:
                        e[1] -= int(tg[s])
                        if e[1] <= 0:
                            done.append(s)
                _, per = p.batch.sync_status(stream=p.stream)
                # a voxel that stopped (trapped, or a numeric error) ends its request too
                done = sorted(set(done) | {s for s in p.active if per[s] != 0})
                for s in done:
                    r, _, adm, ran, work = p.active.pop(s)
                    st = p.batch.read_state(s, stream=p.stream) if collect_state else None
                    results.append(Result(r.rid, r.arrival, adm, tdone, ran, int(per[s]), st,
                                          float(clk[s]) if clk is not None else 0.0, work))
                    p.free.append(s)
        elapsed = time.perf_counter() - t0
        return results, {"elapsed_s": elapsed, "busy_s": busy, "events": total_events, "launches": launches,
                         "events_per_s": total_events / max(elapsed, 1e-9), "slots": self.n_slots,
                         "pools": len(self.pools), "bytes": self.used_bytes}

    def _clocks(self, p):
        host = {"t_hi": np.zeros(p.n, np.float64), "t_lo": np.zeros(p.n, np.float64)}
        p.batch.read_batch_state(host, stream=p.stream)
        if p.stream is not None:
            p.stream.synchronize()
        return host["t_hi"] + host["t_lo"]

    def close(self):
        for p in self.pools:
            p.close()
        self.pools = []


def latency_summary(results: Sequence[Result]):
    lat = np.array([r.latency_per_1e6 for r in results])
    if lat.size == 0:
        return {}
    return {"requests": int(lat.size), "p50_s_per_1e6": float(np.percentile(lat, 50)),
            "p99_s_per_1e6": float(np.percentile(lat, 99)),
            "p50_latency_s": float(np.percentile([r.latency for r in results], 50)),
            "p99_latency_s": float(np.percentile([r.latency for r in results], 99)),
            "makespan_s": float(max(r.finished for r in results))}
