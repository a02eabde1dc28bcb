#!/usr/bin/env python
"""Benchmark: AKMC vacancy-hop events/s on GB300 (batched vs plain) and the
rate-kernel memory bandwidth.

Default workload (one step): the batched EAM configuration -- 256 independent
voxels of 32^3 bcc cells (65,536 sites each), Fe-0.3Cu-0.7Ni-1.4Mn at%, one
vacancy each, synthetic seeded EAM tables, FP32 embedding with exact
fixed-point + FP64 assembly, FP64 rate sums and compensated FP64 clock --
advanced by 1e6 events on every voxel.  Inputs are resident in HBM; the L2
is flushed between timed steps (the 84 MB of lattices and densities would
otherwise stay in the 129 MB L2 between steps).

Also reported: the plain form (Fe-1.34Cu, 16^3 cells, pair model, FP64, one
kernel launch per event) and the persistent one-voxel form; the rate
kernel (akmc_compute_rates: densities + rates + trees) over a working set
larger than L2; an end-to-end number through the public API with host
buffers; the oracle on the host cores (CPU baseline).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank steps its own 256 voxels (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "AKMC vacancy-hop events/sec per GB300 (batched vs plain) + rate-kernel HBM GB/s"
UNIT = "events/s"
N_VOX = 256
# Algorithmic bytes of one EAM event in the step kernel: read the 145-site
# read set (species 1 B + density 4 B each), write the 2 swapped species and
# read+write the densities of the 78 sites the hop changes.
EAM_BYTES_PER_EVENT = 145 * (1 + 4) + 2 + 78 * 4 * 2
# Rate kernel (akmc_compute_rates) algorithmic bytes per site: read species
# (1 B) and write the density (4 B).
RATE_BYTES_PER_SITE = 5
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per event of one
# full-size step-kernel launch, from one ncu capture of
# `bench.py --steps 3 --warmup 3 --no-extras --launch 8,0` (696 MB read +
# 5.39 GB written for 2.56e8 events), and warp instructions per event
# (smsp__inst_executed.sum of the 2000-event case of the same workload);
# valid only for the kernel source they were taken from.
NCU_STEP_TRAFFIC = {"k_step_sha1": "59c1ee62c3adf61a031e4b08f32b3c1e1822b2ed", "bytes_per_event": 23.79,
                    "warp_inst_per_event": 4196}


def _step_src_sha1():
    p = os.path.join(ROOT, "paper_2604_24091_gb300", "csrc", "k_step.cu")
    return hashlib.sha1(open(p, "rb").read()).hexdigest()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi SM clock and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if "Active" in r[5 + k] and "Not" not in r[5 + k]:
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU side

def _oracle_worker(args):
    desc, n_events = args
    import oracle
    v = oracle.Voxel(desc, synth.default_model())
    t0 = time.perf_counter()
    v.step(n_events)
    return n_events, time.perf_counter() - t0


def cpu_oracle_rate(descs, events_per_voxel, procs):
    """The oracle as it stands on `procs` host processes (one voxel each,
    spawned so no process is forked after CUDA initialisation)."""
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(d, events_per_voxel) for d in descs[:procs]])
    ev = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return ev / wall, ev, wall


def workload_name(events_per_voxel):
    return ("batched EAM: %d voxels x 32^3 cells (65536 sites), Fe-0.3Cu-0.7Ni-1.4Mn at%%, 1 vacancy, 563 K, "
            "%d events per voxel per step" % (N_VOX, events_per_voxel))


def reference_arm(args):
    """--impl reference: the oracle timed on the host cores, same metric and
    workload, each step a bounded sample (one voxel per core, fixed events)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    procs = os.cpu_count() or 1
    descs = synth.config_batched_eam(N_VOX)
    per = args.ref_events
    for _ in range(args.warmup):
        cpu_oracle_rate(descs, max(200, per // 50), procs)
    rates, walls, evs = [], [], 0
    for _ in range(args.steps):
        r, ev, wall = cpu_oracle_rate(descs, per, procs)
        rates.append(r)
        walls.append(wall)
        evs += ev
    value = evs / sum(walls)
    sample = "%d of the %d voxels (one per host core), %d events each per step" % (procs, N_VOX, per)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_name(args.events), "voxels_per_gpu": N_VOX,
                       "events_per_voxel_per_step": int(args.events), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU side

def _time_region(fn, torch):
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    fn()
    e.record()
    e.synchronize()
    return s.elapsed_time(e) * 1e-3


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--events", type=int, default=1_000_000, help="events per voxel per step")
    ap.add_argument("--ref-events", type=int, default=100000,
                    help="oracle events per host core per step (reference arm; the cpu_baseline leg runs 3x)")
    ap.add_argument("--no-extras", action="store_true", help="skip plain/e2e/rate-kernel/cpu legs")
    ap.add_argument("--launch", default=None, help="warps,ctas_per_sm of the step kernel (skips the tuner)")
    ap.add_argument("--rate-kernel", action="store_true",
                    help="run only the rate-kernel leg (300 EAM voxels of 64^3 cells) and print its JSON")
    ap.add_argument("--sublattice", action="store_true",
                    help="run only the large-voxel sublattice leg (128^3 cells, 64 vacancies) and print its JSON")
    ap.add_argument("--serving", action="store_true",
                    help="run the serving workload (Poisson arrivals, continuous batching) instead")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.serving:
        return serving(args)
    if args.rate_kernel:
        import torch
        from paper_2604_24091_gb300 import Batch
        torch.cuda.set_device(0)
        peak, peak_kind = _peaks()
        print(json.dumps(rate_kernel_leg(synth.default_model(), torch, peak, peak_kind, Batch)), flush=True)
        return
    if args.sublattice:
        import torch
        from paper_2604_24091_gb300 import Batch
        torch.cuda.set_device(0)
        print(json.dumps(sublattice_leg(synth.default_model(), torch, Batch)), flush=True)
        return

    import torch
    import torch.distributed as dist
    from paper_2604_24091_gb300 import Batch
    from paper_2604_24091_gb300 import shard as S
    from paper_2604_24091_gb300 import tune as T

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    model = synth.default_model()
    descs = synth.config_batched_eam(N_VOX)
    descs = S.rank_descs(descs, rank, lambda uid: synth.splitmix64(synth.SEED_BASE + 2, uid))
    if args.launch:
        warps, per_sm = (int(x) for x in args.launch.split(","))
    else:
        warps, per_sm = T.tune(descs, model, events=3000)
    b = Batch(descs, model)
    b.set_launch(warps, per_sm)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    E = int(args.events)
    n_ev = np.full(N_VOX, E, np.uint64)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        b.step(n_ev)
    st, per = b.sync_status()
    assert st == 0, "voxel status %s" % np.unique(per)
    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    t_wall0 = time.perf_counter()
    times = []
    for _ in range(args.steps):
        flush.zero_()                                   # L2 flush, outside the timed events
        times.append(_time_region(lambda: b.step(n_ev), torch))
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    st, per = b.sync_status()
    assert st == 0, "voxel status %s" % np.unique(per)
    dev_time = S.max_over_ranks(sum(times), dist if world > 1 else None, dev)
    events_total = float(E) * N_VOX * args.steps * world
    value = events_total / dev_time
    peak, peak_kind = _peaks()
    achieved_gbs = EAM_BYTES_PER_EVENT * float(E) * N_VOX * args.steps / sum(times) / 1e9
    traffic, issue = None, None
    if NCU_STEP_TRAFFIC["k_step_sha1"] == _step_src_sha1() and NCU_STEP_TRAFFIC["bytes_per_event"]:
        traffic = NCU_STEP_TRAFFIC["bytes_per_event"] * float(E) * N_VOX
        # instruction-issue roof: 4 schedulers per SM, one warp instruction per cycle each
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_issue = n_sm * 4 * ((clocks or {}).get("sm_max_mhz") or 2070.0) * 1e6
        ach_issue = value / world * NCU_STEP_TRAFFIC["warp_inst_per_event"]
        issue = {"warp_inst_per_event": NCU_STEP_TRAFFIC["warp_inst_per_event"], "achieved": ach_issue,
                 "peak": peak_issue, "unit": "warp instructions/s", "frac": ach_issue / peak_issue}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_time / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (EAM split: FP32 embedding, exact "
        "fixed-point + FP64 assembly, FP64 rate sums and clock)", "data": "synthetic",
        "config": {"workload": workload_name(E),
                   "voxels_per_gpu": N_VOX, "events_per_voxel_per_step": E, "launch": [warps, per_sm],
                   "l2": "flushed between timed steps (256 MB write)", "wall_s_timed_region": t_wall},
        "roofline": {"bound": "hbm", "kernel": "step_kernel (persistent, one CTA per voxel)",
                     "achieved": achieved_gbs, "peak": peak, "unit": "GB/s", "frac": achieved_gbs / peak,
                     "traffic": traffic, "peak_kind": peak_kind,
                     "bytes_per_event": EAM_BYTES_PER_EVENT, "issue": issue,
                     "note": "latency-bound: each voxel is one serial event chain"},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_extras:
        line.update(extras(b, descs, model, torch, dev, n_ev, args, peak, peak_kind, Batch))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def rate_kernel_leg(model, torch, peak, peak_kind, Batch):
    """akmc_compute_rates (densities + rates + trees) over a working set
    larger than L2: 300 EAM voxels of 64^3 cells (157 M sites: 157 MB species
    + 629 MB densities).  Best of 5 launches."""
    big = [synth.VoxelDesc(64, 2, (0.002, 0.01, 0.01), 563.0, synth.EAM_MODEL, synth.PREC_SPLIT,
                           synth.splitmix64(99, u), u) for u in range(300)]
    rb = Batch(big, model)
    rb.compute_rates()
    ts = [_time_region(rb.compute_rates, torch) for _ in range(5)]
    sites = sum(2 * d.L ** 3 for d in big)
    gbs = RATE_BYTES_PER_SITE * sites / min(ts) / 1e9
    rb.close()
    return {"bound": "hbm", "kernel": "akmc_compute_rates (density + rates + trees)",
            "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "traffic": None, "peak_kind": peak_kind,
            "workload": "300 EAM voxels x 64^3 cells, 157 M sites (> L2)",
            "ms": 1e3 * min(ts)}


def logit_select_leg(torch, dev, peak, peak_kind):
    """Global masked softmax sampling (akmc_select_logits) over 256 systems of
    65536 agents x 8 candidate transitions (134 M float32 logits + uint8 mask,
    671 MB > L2); algorithmic bytes 5 per logit (each logit and mask byte read
    once).  Best of 5 calls."""
    from paper_2604_24091_gb300 import SelectPlan, select_logits
    n_seg, per = 256, 65536 * 8
    g = torch.Generator(device=dev)
    g.manual_seed(synth.SEED_BASE + 6)
    logits = torch.randn(n_seg * per, generator=g, device=dev, dtype=torch.float32) * 2.0
    mask = (torch.rand(n_seg * per, generator=g, device=dev) < 0.02).to(torch.uint8)
    plan = SelectPlan(np.arange(n_seg + 1, dtype=np.int64) * per)
    select_logits(plan, logits, 1.0, 1, 0, mask)
    ts = [_time_region(lambda c=c: select_logits(plan, logits, 1.0, 1, c + 1, mask), torch) for c in range(5)]
    gbs = 5.0 * n_seg * per / min(ts) / 1e9
    return {"bound": "hbm", "kernel": "akmc_select_logits (part pass, system search)", "achieved": gbs,
            "peak": peak, "unit": "GB/s", "frac": gbs / peak, "traffic": None, "peak_kind": peak_kind,
            "workload": "256 systems x 524288 logits (float32) + mask (uint8), 671 MB", "ms": 1e3 * min(ts)}


def sublattice_leg(model, torch, Batch, sector_cells=16, n_st=800, windows=(1.0, 4.0)):
    """The large configuration (128^3 cells, 64 vacancies, EAM split) under
    sublattice supersteps, synchronous (one launch per superstep) and
    asynchronous (one launch, per-sector readiness): sectors of 16 cells, windows
    sized for f events per active vacancy.  The yield is the events made over
    the events the global rate makes in the same voxel time (R_tot T/8 per
    superstep): what the octant boundaries cost."""
    cfg = synth.config_large()
    out = {"config": "1 voxel of 128^3 cells, 64 vacancies, EAM split, sectors of %d cells, %d supersteps"
                     % (sector_cells, n_st)}
    for f in windows:
        for form in ("sync", "async"):
            lb = Batch(cfg, model)
            r_tot = float(lb.read_state(0)["rates"].sum())
            T = f / (r_tot / cfg[0].n_vac)
            asy = form == "async"
            lb.step_sublattice(0, 0, 16, sector_cells, T, asynchronous=asy)
            n0 = lb.read_state(0)["n_events"]
            t = _time_region(lambda: lb.step_sublattice(0, 16, n_st, sector_cells, T, asynchronous=asy), torch)
            st, _ = lb.sync_status()
            made = lb.read_state(0)["n_events"] - n0
            out["%s_f%g" % (form, f)] = {"value": made / t, "unit": UNIT, "status": st, "window_s": T,
                                         "events_per_superstep": made / n_st, "supersteps_per_s": n_st / t,
                                         "yield": made / (n_st * r_tot * T / 8)}
            lb.close()
    return out


def extras(b, descs, model, torch, dev, n_ev, args, peak, peak_kind, Batch):
    out = {}
    # end to end through the public API with pinned host buffers: load the
    # lattices, (rebuild), step, read the lattices and clocks back
    host = b.host_buffers(pinned=True)
    b.read_batch_state(host)
    torch.cuda.synchronize()
    h2d = host["species"].nbytes + host["vac_pos"].nbytes + 3 * 8 * b.n
    d2h = (host["species"].nbytes + host["vac_pos"].nbytes + host["vac_disp"].nbytes + 3 * 8 * b.n + 4 * b.n)
    e2e_times = []
    for i in range(max(1, args.steps)):
        t0 = time.perf_counter()
        b.load_batch_state(host["species"], host["vac_pos"], host["t_hi"], host["t_lo"], host["n_events"])
        b.step(n_ev)
        b.read_batch_state(host)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        assert (host["status"] == 0).all()
    out["e2e"] = {"value": float(n_ev.sum()) * len(e2e_times) / sum(e2e_times), "unit": UNIT,
                  "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                  "api": "load_batch_state -> step_n -> read_batch_state, pinned host buffers"}
    # plain form: Fe-1.34Cu 16^3 pair model FP64, one launch per event; and the
    # same voxel under one persistent launch
    c1 = synth.config_plain_pair()
    p = Batch(c1, model)
    p.set_launch(4, 0)
    one = np.ones(1, np.uint64)
    for _ in range(50):
        p.step(one)
    n_plain = 3000
    t = _time_region(lambda: [p.step(one) for _ in range(n_plain)], torch)
    n_pers = 100000
    tp = _time_region(lambda: p.step(np.full(1, n_pers, np.uint64)), torch)
    out["plain"] = {"value": n_plain / t, "unit": UNIT,
                    "config": "Fe-1.34Cu 16^3 cells pair model FP64, 1 voxel, one kernel launch per event",
                    "persistent_one_voxel": n_pers / tp}
    p.close()
    out["rate_kernel_roofline"] = rate_kernel_leg(model, torch, peak, peak_kind, Batch)
    out["logit_select_roofline"] = logit_select_leg(torch, dev, peak, peak_kind)
    # the uneven configuration (1000 voxels, L 16-64, 1-8 vacancies, pair/EAM)
    # and the large one (128^3 cells, 64 vacancies): events/s of one persistent launch
    for key, cfg, per_vac in (("uneven", synth.config_uneven(1000), 10000), ("large", synth.config_large(), 20000)):
        ub = Batch(cfg, model)
        tg = np.array([per_vac * d.n_vac for d in cfg], np.uint64) if key == "uneven" else \
            np.full(len(cfg), per_vac, np.uint64)
        ub.step(np.minimum(tg, 200).astype(np.uint64))
        tu = _time_region(lambda: ub.step(tg), torch)
        stu, _ = ub.sync_status()
        extra = {}
        if key == "large":   # the Cu-cluster histogram taken every 1e6 events of this configuration
            ub.cluster_hist(0)
            th = []
            for _ in range(3):
                t0 = time.perf_counter()
                ub.cluster_hist(0)
                th.append(time.perf_counter() - t0)
            extra = {"cluster_hist_ms": 1e3 * min(th), "events_between_histograms": 1000000}
        out[key] = {"value": float(tg.sum()) / tu, "unit": UNIT, "status": stu, **extra,
                    "config": ("1000 voxels, L in {16,24,32,48,64}, 1-8 vacancies, pair/EAM 50/50, "
                               "1e4 events per vacancy" if key == "uneven" else
                               "1 voxel of 128^3 cells, 64 vacancies, EAM split, 2e4 events")}
        ub.close()
    out["large_sublattice"] = sublattice_leg(model, torch, Batch)
    # the oracle on the host cores, bounded sample of the same workload
    procs = os.cpu_count() or 1
    per = 3 * args.ref_events
    r, ev, wall = cpu_oracle_rate(descs, per, procs)
    out["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": procs, "kind": "oracle",
                           "sample": "%d voxels of the workload, one per host core, %d events each (%.1f s)"
                           % (procs, per, wall)}
    return out


def serving(args):
    """Serving workload: Poisson arrivals (200 requests/s for 10 s) of
    batched-EAM-like voxels (32^3 cells, 1 vacancy, split precision), each
    asking for 1e6-1e7 events (log-uniform), admitted under a 120 GB HBM
    budget with continuous batching; then the same at 70% of the measured
    capacity.  Reports p50/p99 latency per 1e6 events and events/s."""
    import torch
    from paper_2604_24091_gb300.serve import Request, Server, latency_summary
    torch.cuda.set_device(0)
    model = synth.default_model()
    shape = synth.VoxelDesc(32, 1, (0.003, 0.007, 0.014), 563.0, synth.EAM_MODEL, synth.PREC_SPLIT)
    srv = Server(model, shape, hbm_budget=120e9, max_slots=2048, chunk=20000)
    out = {"metric": METRIC + " (serving)", "unit": UNIT, "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "serving: Poisson 200 req/s for 10 s, 32^3-cell EAM voxels, 1e6-1e7 events "
                      "each, 120 GB HBM budget", "slots": srv.n_slots, "bytes_per_slot": srv.bytes_per_slot,
                      "chunk_events": srv.chunk}}
    reqs = [Request(t, d, n, i) for i, (t, d, n) in enumerate(synth.serving_requests(10.0, 200.0))]
    res, st = srv.run(reqs)
    out["window"] = dict(latency_summary(res), events_per_s=st["events_per_s"], elapsed_s=st["elapsed_s"],
                         requests_offered=len(reqs), offered_events=int(sum(r.n_events for r in reqs)))
    cap = st["events"] / max(st["busy_s"], 1e-9)
    mean_ev = float(np.mean([r.n_events for r in reqs]))
    lam = 0.7 * cap / mean_ev
    reqs70 = [Request(t, d, n, i) for i, (t, d, n) in
              enumerate(synth.serving_requests(10.0, lam, seed=synth.SEED_BASE + 15))]
    res70, st70 = srv.run(reqs70)
    out["at_70pct_capacity"] = dict(latency_summary(res70), events_per_s=st70["events_per_s"],
                                    rate_hz=lam, requests=len(reqs70), capacity_events_per_s=cap)
    # the same requests in FP64 EAM (the reference precision; split-mode energy changes agree with it
    # within 1e-5 eV): capacity from a saturated offline batch, then arrivals at 70 % of it
    shape64 = dataclasses.replace(shape, precision=synth.PREC_FP64)
    srv64 = Server(model, shape64, hbm_budget=120e9, max_slots=2048, chunk=20000)
    probe = [Request(0.0, dataclasses.replace(d, precision=synth.PREC_FP64), 200000, i)
             for i, (t, d, n) in enumerate(synth.serving_requests(10.0, 200.0, seed=synth.SEED_BASE + 16)[:srv64.n_slots])]
    _, stp = srv64.run(probe, realtime=False)
    cap64 = stp["events"] / max(stp["busy_s"], 1e-9)
    lam64 = 0.7 * cap64 / mean_ev
    reqs64 = [Request(t, d, n, i) for i, (t, d, n) in
              enumerate(synth.serving_requests(10.0, lam64, seed=synth.SEED_BASE + 15, precision=synth.PREC_FP64))]
    res64, st64 = srv64.run(reqs64)
    out["fp64_at_70pct_capacity"] = dict(latency_summary(res64), events_per_s=st64["events_per_s"], rate_hz=lam64,
                                         requests=len(reqs64), capacity_events_per_s=cap64)
    out["value"] = st["events_per_s"]
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
