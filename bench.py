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
# `bench.py --steps 3 --warmup 3 --no-extras --launch 8,0` (0.687 GB read +
# 5.291 GB written for 2.56e8 events), and warp instructions per event
# (smsp__inst_executed.sum 1.949e9 of the 2000-event case of the same workload);
# valid only for the kernel source they were taken from.
NCU_STEP_TRAFFIC = {"k_step_sha1": "999ac0a3ea624035118fbafb4dfe50ac29eecebe", "bytes_per_event": 23.35,
                    "warp_inst_per_event": 3807}


# DRAM bytes of one density_strip_kernel launch on the rate-kernel workload (300
# EAM voxels of 64^3 cells): 167 MB read + 569 MB written, from one ncu capture
# of `bench.py --rate-kernel`; valid only for the kernel source it was taken from.
NCU_RATE_TRAFFIC = {"k_density_sha1": "0c17618c42557127bfeb82c64bc81b39125d1dc3", "bytes": 736.4e6}


def _src_sha1(name):
    p = os.path.join(ROOT, "paper_2604_24091_gb300", "csrc", name)
    return hashlib.sha1(open(p, "rb").read()).hexdigest()


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
    ap.add_argument("--large-run", action="store_true",
                    help="run the large configuration as configured (128^3 cells, 64 vacancies, 1e8 events, "
                         "Cu-cluster histogram every 1e6 events) and print its JSON")
    ap.add_argument("--large-events", type=int, default=100_000_000, help="events of --large-run")
    ap.add_argument("--large-every", type=int, default=1_000_000,
                    help="events between Cu-cluster histograms in --large-run (one step launch each)")
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
    if args.large_run:
        import torch
        from paper_2604_24091_gb300 import Batch
        torch.cuda.set_device(0)
        print(json.dumps(large_run(synth.default_model(), torch, Batch, args.large_events, args.large_every)),
              flush=True)
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
        # The step kernel's roof is instruction issue (each voxel is one serial event
        # chain; its 84 MB working set stays in L2): achieved warp instructions/s
        # against 4 schedulers per SM at the SM clock.  The HBM fraction is kept
        # beside it for the contract's algorithmic-bytes view.
        "roofline": dict(
            ({"bound": "alu", "achieved": issue["achieved"], "peak": issue["peak"], "unit": issue["unit"],
              "frac": issue["frac"], "warp_inst_per_event": issue["warp_inst_per_event"],
              "peak_kind": "152 SMs x 4 schedulers x max SM clock, one warp instruction per cycle each"}
             if issue else {"bound": "alu", "achieved": None, "peak": None, "unit": "warp instructions/s",
                            "frac": None}),
            kernel="step_kernel (persistent, one CTA per voxel)", traffic=traffic,
            hbm={"achieved": achieved_gbs, "peak": peak, "unit": "GB/s", "frac": achieved_gbs / peak,
                 "peak_kind": peak_kind, "bytes_per_event": EAM_BYTES_PER_EVENT, "traffic": traffic},
            note="latency- and issue-bound: each voxel is one serial event chain; DRAM carries ~24 B/event"),
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_extras:
        line.update(extras(b, descs, model, torch, dev, n_ev, args, peak, peak_kind, Batch, (warps, per_sm)))
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
    traffic = NCU_RATE_TRAFFIC["bytes"] if _src_sha1("k_density.cu") == NCU_RATE_TRAFFIC["k_density_sha1"] else None
    return {"bound": "hbm", "kernel": "akmc_compute_rates (density + rates + trees)",
            "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "traffic": traffic, "algorithmic_bytes": RATE_BYTES_PER_SITE * sites, "peak_kind": peak_kind,
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


def large_run(model, torch, Batch, total=100_000_000, every=1_000_000):
    """The large configuration as configured: one voxel of 128^3 cells
    (4.19 M sites), 64 vacancies, EAM split precision, global residence-time
    selection over the device-resident rate tree, run to 1e8 events with the
    Cu-cluster size histogram (1nn+2nn) taken every 1e6 events.  Events/s
    counts the stepping time only (CUDA events); the histograms are timed
    apart."""
    cfg = synth.config_large()
    lb = Batch(cfg, model)
    t_step, t_hist, series, clock = 0.0, 0.0, [], []
    wall0 = time.perf_counter()
    for k in range(total // every):
        t_step += _time_region(lambda: lb.step(every), torch)
        t0 = time.perf_counter()
        series.append(lb.cluster_hist(0).tolist())
        t_hist += time.perf_counter() - t0
        st = lb.read_state(0, species=False)
        clock.append(st["t_hi"] + st["t_lo"])
        # one progress line per histogram (stderr), so a cut-off run keeps its series
        sys.stderr.write(json.dumps({"events": st["n_events"], "step_seconds": t_step, "clock_s": clock[-1],
                                     "hist": series[-1], "status": st["status"]}) + "\n")
        sys.stderr.flush()
        if st["status"] != 0:
            break
    s = lb.read_state(0, species=False)
    lb.close()
    return {"config": "1 voxel of 128^3 cells (4194304 sites), Fe-0.2Cu-0.7Ni-1.4Mn at%%, 64 vacancies, EAM split, "
                      "%d events, Cu-cluster histogram every %d events" % (total, every),
            "events": s["n_events"], "status": s["status"], "value": s["n_events"] / t_step, "unit": UNIT,
            "step_seconds": t_step, "histogram_ms_mean": 1e3 * t_hist / max(1, len(series)),
            "wall_s": time.perf_counter() - wall0, "simulated_time_s": clock[-1] if clock else 0.0,
            "bins": "1,2,3,4,5-9,10-19,20-49,>=50", "histograms": series, "clock_s": clock}


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


def split_vs_fp64(model, Batch, pairs):
    """Largest |dE_split - dE_fp64| (eV) and relative rate difference over GPU
    states of split-precision EAM voxels: every (descriptor, state) pair is
    loaded into a float64-EAM batch on the GPU (akmc_load_state, then
    akmc_compute_rates) and the 8 hop energy changes of every vacancy compared."""
    if not pairs:
        return None
    fd = [dataclasses.replace(d, precision=synth.PREC_FP64) for d, _ in pairs]
    fb = Batch(fd, model)
    for i, (_, s) in enumerate(pairs):
        fb.load_state(i, s["species"], s["vac_pos"], s["t_hi"], s["t_lo"], s["n_events"])
    fb.compute_rates()
    de, rr, hops = 0.0, 0.0, 0
    for i, (_, s) in enumerate(pairs):
        f = fb.read_state(i, species=False)
        de = max(de, float(np.abs(f["dE"] - s["dE"]).max()))
        m = f["rates"] > 0
        if m.any():
            rr = max(rr, float((np.abs(f["rates"][m] - s["rates"][m]) / f["rates"][m]).max()))
        hops += int(f["dE"].size)
    fb.close()
    return {"max_abs_dE_eV": de, "max_rel_rate_diff": rr, "voxels": len(pairs), "hops": hops,
            "tolerance_eV": 1e-5, "reference": "float64 EAM path on the GPU (= float64 oracle within 1e-12 eV)"}


def uneven_leg(model, torch, Batch, per_vac=100000, replays=10):
    """The uneven configuration as configured: 1000 voxels, 1e5 events per
    vacancy, launch shape from the autotuner, advanced by `replays` replays of
    one captured CUDA graph (each replay: per_vac / replays events per vacancy)."""
    from paper_2604_24091_gb300 import tune as T
    cfg = synth.config_uneven(1000)
    t0 = time.perf_counter()
    shape = T.tune(cfg, model, events=2000)
    t_tune = time.perf_counter() - t0
    ub = Batch(cfg, model)
    ub.set_launch(*shape)
    ub.step(np.array([200 * d.n_vac for d in cfg], np.uint64))   # warm-up (not counted)
    chunk = np.array([per_vac // replays * d.n_vac for d in cfg], np.uint64)
    g = ub.capture_step(chunk)
    torch.cuda.synchronize()
    tu = _time_region(lambda: [g.replay() for _ in range(replays)], torch)
    stu, _ = ub.sync_status()
    n = float(chunk.sum()) * replays
    return {"value": n / tu, "unit": UNIT, "status": stu, "events": n, "seconds": tu,
            "launch": list(shape), "tune_s": t_tune, "graph_replays": replays,
            "config": "1000 voxels, L in {16,24,32,48,64}, 1-8 vacancies, pair/EAM 50/50, T 543-593 K, "
                      "1e5 events per vacancy, autotuned launch shape, CUDA-graph replays"}, ub


def extras(b, descs, model, torch, dev, n_ev, args, peak, peak_kind, Batch, launch):
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
    # the uneven configuration as configured: 1000 voxels (L 16-64, 1-8 vacancies,
    # pair/EAM mixed), 1e5 events per vacancy, the autotuner's launch shape, run as
    # replays of one captured CUDA graph (10 replays of 1e4 events per vacancy)
    out["uneven"], ub = uneven_leg(model, torch, Batch)
    # the large configuration (128^3 cells, 64 vacancies): events/s of one persistent launch
    lcfg = synth.config_large()
    lb = Batch(lcfg, model)
    lb.step(200)
    tl = _time_region(lambda: lb.step(20000), torch)
    stl, _ = lb.sync_status()
    lb.cluster_hist(0)
    th = []
    for _ in range(3):
        t0 = time.perf_counter()
        lb.cluster_hist(0)
        th.append(time.perf_counter() - t0)
    out["large"] = {"value": 20000 / tl, "unit": UNIT, "status": stl, "cluster_hist_ms": 1e3 * min(th),
                    "events_between_histograms": 1000000,
                    "config": "1 voxel of 128^3 cells, 64 vacancies, EAM split, 2e4 events (the full 1e8-event "
                              "run with a histogram every 1e6 events: bench.py --large-run)"}
    # precision: split-precision EAM against the float64 EAM path, per configuration,
    # on sampled GPU states (the float64 path matches the float64 oracle within 1e-12 eV)
    prec = {}
    sample = [0, 37, 101, 150, 203, 255]
    prec["batched_eam"] = split_vs_fp64(model, Batch, [(descs[v], b.read_state(v)) for v in sample])
    eam_u = [v for v, d in enumerate(ub.descs) if d.model == synth.EAM_MODEL][:24]
    prec["uneven_eam"] = split_vs_fp64(model, Batch, [(ub.descs[v], ub.read_state(v)) for v in eam_u])
    prec["large"] = split_vs_fp64(model, Batch, [(lcfg[0], lb.read_state(0))])
    ub.close()
    lb.close()
    # the batched workload in float64 EAM: events/s beside the split precision
    f64 = Batch(synth.config_batched_eam(N_VOX, precision=synth.PREC_FP64), model)
    f64.set_launch(*launch)
    f64.step(2000)
    n64 = 100000
    t64 = _time_region(lambda: f64.step(n64), torch)
    st64, _ = f64.sync_status()
    prec["batched_eam_fp64_events_per_s"] = {"value": n64 * N_VOX / t64, "unit": UNIT, "status": st64,
                                             "events_per_voxel": n64}
    f64.close()
    out["precision"] = prec
    out["large_sublattice"] = sublattice_leg(model, torch, Batch)
    out["serving"], out["precision"]["serving"] = serving_block(model, torch, Batch)
    # the oracle on the host cores, bounded sample of the same workload
    procs = os.cpu_count() or 1
    per = 3 * args.ref_events
    r, ev, wall = cpu_oracle_rate(descs, per, procs)
    out["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": procs, "kind": "oracle",
                           "sample": "%d voxels of the workload, one per host core, %d events each (%.1f s)"
                           % (procs, per, wall)}
    return out


def _serve_window(model, torch, duration, policy, rate=200.0, seed=None, precision=None, reserve_slots=2048,
                  collect_state=False):
    """Config-5 Poisson window: arrivals at `rate` for `duration` s of 32^3-cell
    EAM requests (1e6-1e7 events each), 120 GB budget, one reserved pool."""
    from paper_2604_24091_gb300.serve import Request, Server, latency_summary
    prec = synth.PREC_SPLIT if precision is None else precision
    proto = synth.VoxelDesc(32, 1, (0.003, 0.007, 0.014), 563.0, synth.EAM_MODEL, prec)
    srv = Server(model, hbm_budget=120e9, chunk=20000, policy=policy, reserve=[(proto, reserve_slots)])
    kw = {} if seed is None else {"seed": seed}
    reqs = [Request(t, d, n, i) for i, (t, d, n) in
            enumerate(synth.serving_requests(duration, rate, precision=prec, **kw))]
    res, st = srv.run(reqs, collect_state=collect_state)
    for r in res:
        r.desc = reqs[r.rid].desc
    out = dict(latency_summary(res), events_per_s=st["events_per_s"], elapsed_s=st["elapsed_s"],
               requests_offered=len(reqs), offered_events=int(sum(r.n_events for r in reqs)),
               slots=srv.n_slots, capacity_events_per_s=st["events"] / max(st["busy_s"], 1e-9),
               statuses=sorted({r.status for r in res}))
    srv.close()
    return out, res


def serving_ensemble(model, torch, policy, n=384, slots_budget=48e6):
    """The dynamic voxel scheduling claim (Eq. 10): an ensemble of mixed-shape
    voxels, each advanced by a simulated-time horizon, all due at once, more
    requests than slots (HBM budget); makespan and latency with FIFO admission
    or largest expected work (nu W0 t_sim) first."""
    from paper_2604_24091_gb300.serve import Request, Server, latency_summary
    reqs = [Request(0.0, d, t_sim=t, rid=i) for i, (d, t) in enumerate(synth.mixed_requests(n))]
    srv = Server(model, hbm_budget=slots_budget, chunk=50000, policy=policy, min_pool=8, max_pool=64)
    res, st = srv.run(reqs, realtime=False)
    out = dict(latency_summary(res), events=st["events"], events_per_s=st["events_per_s"],
               elapsed_s=st["elapsed_s"], pools=st["pools"], bytes=st["bytes"], requests=len(reqs),
               statuses=sorted({r.status for r in res}))
    srv.close()
    return out, res


def serving_block(model, torch, Batch):
    """Serving in the default bench line: a 1-s config-5 Poisson window with
    FIFO and with proxy admission (p50/p99 per 1e6 events), the mixed-shape
    time-horizon ensemble with both policies, and the split-precision error
    of served results against the float64 EAM path."""
    out = {}
    for pol in ("fifo", "proxy"):
        out["window_1s_" + pol], res = _serve_window(model, torch, 1.0, pol, collect_state=pol == "fifo")
        if pol == "fifo":
            sample = [r for r in res if r.state is not None][:8]
            prec = split_vs_fp64(model, Batch, [(r.desc, r.state) for r in sample])
    out["ensemble_fifo"], _ = serving_ensemble(model, torch, "fifo")
    out["ensemble_proxy"], _ = serving_ensemble(model, torch, "proxy")
    return out, prec


def serving(args):
    """Serving workload (config 5): Poisson arrivals (200 requests/s for 10 s)
    of batched-EAM-like voxels (32^3 cells, 1 vacancy, split precision), each
    asking for 1e6-1e7 events (log-uniform), admitted under a 120 GB HBM
    budget with continuous batching; then the same at 70% of the measured
    capacity, FIFO and proxy admission; the same requests in float64 EAM at
    70% of its own capacity; and the mixed-shape ensemble.  Reports p50/p99
    latency per 1e6 events and events/s."""
    import torch
    from paper_2604_24091_gb300 import Batch
    torch.cuda.set_device(0)
    model = synth.default_model()
    out = {"metric": METRIC + " (serving)", "unit": UNIT, "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "serving: Poisson 200 req/s for 10 s, 32^3-cell EAM voxels, 1e6-1e7 events "
                      "each, 120 GB HBM budget"}}
    out["window"], res = _serve_window(model, torch, 10.0, "fifo")
    cap = out["window"]["capacity_events_per_s"]
    mean_ev = 5.5e6
    lam = 0.7 * cap / mean_ev
    for pol in ("fifo", "proxy"):
        out["at_70pct_capacity_" + pol], _ = _serve_window(model, torch, 10.0, pol, rate=lam, seed=synth.SEED_BASE + 15)
    # float64 EAM: capacity from a saturated window, then arrivals at 70 % of it
    w64, _ = _serve_window(model, torch, 2.0, "fifo", precision=synth.PREC_FP64)
    cap64 = w64["capacity_events_per_s"]
    out["fp64_at_70pct_capacity"], _ = _serve_window(model, torch, 10.0, "fifo", rate=0.7 * cap64 / mean_ev,
                                                     seed=synth.SEED_BASE + 15, precision=synth.PREC_FP64)
    out["fp64_at_70pct_capacity"]["capacity_events_per_s"] = cap64
    for pol in ("fifo", "proxy"):
        out["ensemble_" + pol], _ = serving_ensemble(model, torch, pol)
    out["value"] = out["window"]["events_per_s"]
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
