#!/usr/bin/env python
"""Throughput benchmark of the GB300 Maxwell-Bloch FDTD hot path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--workload NAME]

One "step" is one time step n -> n+1 of every realization in the workload
(H and E updates with CPML, sources, gain polarization / populations / noise,
probes and flux).  Metric: Mcell-updates/s = sum over realizations of
cells x steps / time.  Prints ONE JSON line on rank 0.

Under torchrun each rank steps its own realizations (different disorder
seeds) with no collective on the data path (weak scaling); the timed region is
bracketed by barriers and the max over ranks is reported.

Besides the headline workload, the default single-GPU run (rank 0) adds:
  * ``batch``: the 64-realization mixed batch (half lasing) stepped together,
    with its roofline fraction and its realizations/hour against the plain
    single-run FP64 GPU path;
  * ``lasing``: the 140^3 Maxwell-Bloch lasing workload, with its roofline
    fraction;
  * ``serve``: a Poisson request stream of the served workload's sizes;
  * ``cpu_baseline``: the FP64 oracle timed on the host cores, one process
    per allowed core (independent realizations) and single-threaded;
  * ``oracle_error``: the GPU path's relative L2 errors against the oracle on
    reduced copies of the workload (and of batch members), computed by the
    same CPU leg.

--impl reference times the FP64 CPU oracle (the reference the library is checked against) on a
bounded sample of the same workload, on the host cores (one process per
allowed core, each stepping its own realization), rank 0 only.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0802_3775_gb300 import inputs  # noqa: E402

METRIC = "Mcell-updates/s"


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------- workloads
NCELL = {"planewave": 8, "lasing": 6}  # unit cells per edge of the workloads (--ncell shrinks them for profiling)


def workload_specs(name: str, rank: int, steps: int):
    """Run records of one rank's share of the workload."""
    if name == "planewave":
        # 8x8x8 unit cells at 20 cells/a + 12-cell CPML = 184^3, FP32, sigma 6 %
        return [inputs.opal_planewave_f32(ncell=NCELL["planewave"], res=20, npml=12, sigma=0.06, realization=rank,
                                          steps=steps)]
    if name == "lasing":
        # 6x6x6 unit cells at 20 cells/a + 10-cell CPML = 140^3, FP32 gain
        return [inputs.opal_lasing_f32(ncell=NCELL["lasing"], res=20, npml=10, sigma=0.05, pump=1e10,
                                       realization=rank, steps=steps)]
    if name == "dipole64":
        return [inputs.opal_dipole_f64(steps=steps)]
    if name == "batch":
        # 64 mixed-size realizations, half passive, half lasing (one launch per step)
        return inputs.mixed_batch(64, seed=4000 + 1000 * rank, steps=steps)
    if name == "planewave64":
        return [inputs.opal_planewave_f32(ncell=8, res=20, npml=12, sigma=0.06, realization=rank, steps=steps,
                                          precision="f64")]
    raise SystemExit(f"unknown workload {name}")


def reduced_specs(name: str, steps: int):
    """Reduced copies of a workload's recipe for the error checks against the
    oracle: 2x2x2 unit cells, the same resolution, absorber, disorder, seeds,
    sources and observers; for the batch its first four members (two passive,
    two lasing) reduced the same way."""
    if name == "planewave":
        return [inputs.opal_planewave_f32(ncell=2, res=20, npml=12, sigma=0.06, realization=0, steps=steps)]
    if name == "planewave64":
        return [inputs.opal_planewave_f32(ncell=2, res=20, npml=12, sigma=0.06, realization=0, steps=steps,
                                          precision="f64")]
    if name == "lasing":
        return [inputs.opal_lasing_f32(ncell=2, res=20, npml=10, sigma=0.05, pump=1e10, realization=0,
                                       steps=steps)]
    if name == "dipole64":
        return [inputs.opal_dipole_f64(steps=steps)]
    if name == "batch":
        return inputs.mixed_batch(4, seed=4000, steps=steps, ncell=2)
    raise SystemExit(f"unknown workload {name}")


WORKLOAD_TEXT = {
    "planewave": "passive disordered fcc inverted opal, 8x8x8 unit cells at 20 cells/a + 12-cell CPML (184^3), "
                 "FP32, sigma 6%, [111] plane-wave Gaussian pulse f=0.80 bw 0.1, FP64 flux plane, 8 probes",
    "lasing": "Maxwell-Bloch lasing opal, 6x6x6 unit cells at 20 cells/a + 10-cell CPML (140^3), FP32, four-level "
              "gain in spheres, pump 1e10/s, noise 1e-6, 6-face flux box, 8 probes",
    "dipole64": "passive fcc opal 2x2x2 unit cells at 12 cells/a + 8-cell CPML (40^3), FP64, Ez dipole pulse",
    "planewave64": "as planewave but FP64 (plain single-run FP64 GPU path)",
    "batch": "64 disorder realizations of mixed size (4^3..8^3 unit cells at 16..20 cells/a + 12-cell CPML, "
             "sigma U(0,10%)), even ones passive [111] plane-wave runs, odd ones four-level lasing runs, FP32, "
             "all stepped together: per time step one launch of each step kernel in use over its members' work items",
}


def algorithmic_bytes(spec, gain_cells: int) -> float:
    """Compulsory HBM bytes of one step-kernel launch: every state word read
    once and written once, material read once."""
    w = 4 if spec.precision == "f32" else 8
    nx, ny, nz = spec.shape
    ncell = nx * ny * nz
    b = ncell * (12 * w + 1)
    n3 = (nx, ny, nz)
    for d in range(3):
        slab = spec.npml[2 * d] + spec.npml[2 * d + 1]
        b += slab * (ncell // n3[d]) * 8 * w
    if spec.gain is not None:
        b += gain_cells * (21 if w == 4 else 15) * w
    return float(b)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return self.summarize(out)

    @staticmethod
    def summarize(out: str):
        """Median SM clock under load, the maximum clock and the throttle
        reasons seen, from nvidia-smi's csv rows (noheader, nounits)."""
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), active=parts[4], hw=parts[5], hwt=parts[6],
                                 swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        smax = max(r["smax"] for r in rows)
        load = [r["sm"] for r in rows if r["sm"] > 0.3 * smax] or [r["sm"] for r in rows]
        reasons = set()
        for r in rows:
            if r["hw"] == "Active":
                reasons.add("hw_slowdown")
            if r["hwt"] == "Active":
                reasons.add("hw_thermal_slowdown")
            if r["swt"] == "Active":
                reasons.add("sw_thermal_slowdown")
            if r["pcap"] == "Active":
                reasons.add("sw_power_cap")
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(rows)}


# ----------------------------------------------------------------------------- ranks
def rank_max(x: float, dist, device: str = "cuda") -> float:
    """Maximum of a per-rank time over all ranks (the job is as slow as its
    slowest replica); x itself when running alone."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- GPU arm
def configure_grid(args, g):
    if args.kernel != "auto":
        g.set_kernel(args.kernel)
    if args.order:
        g.set_item_order(args.order)
    if args.by or args.zdepth:
        g.set_launch(32, args.by, args.zdepth, 0)


def configure_batch(args, b):
    if args.kernel != "auto" or args.by or args.zdepth:
        b.set_launch(args.kernel, args.by, args.zdepth, 0)


KERNEL_NAMES = {1: "k_step", 2: "k_step_tma", 3: "k_step_pair", 4: "k_upml_h + k_upml_e"}


def timed_workload(args, specs, world, dist, steps, warmup, sample_clocks=True):
    """Create the grids of `specs` (a batch when there are several), tune the
    launch shape, warm up, and time `steps` steps with CUDA events on the
    stream the kernels run on.  Returns (record, grids, stepper)."""
    import torch

    from paper_0802_3775_gb300.fdtd import Batch, Grid

    cap = steps + warmup + 16
    grids = [Grid.from_spec(s, record_capacity=cap) for s in specs]
    for g in grids:
        configure_grid(args, g)
    gain_cells = [int(np.count_nonzero(g.get_material() & 64)) if s.gain is not None else 0
                  for g, s in zip(grids, specs)]
    if len(grids) > 1:
        stepper = Batch(grids)
        configure_batch(args, stepper)
    else:
        stepper = grids[0]
    tune = None
    if not args.no_autotune and args.kernel == "auto" and not args.by and not args.zdepth and not args.order:
        # launch shape picked by timing the candidates on this workload (state restored)
        # trials long enough that run-to-run noise does not pick the shape
        # (single grids: 12 shapes x 42 steps, about 60 ms on the 184^3 grid)
        tune = stepper.autotune(trial_steps=40 if len(grids) == 1 else 8)
    stepper.step(warmup)
    stepper.sync()

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.current_stream()
    # CUDA events around every 8th step-kernel launch of the timed region
    # (bracketing every launch costs a few per cent of the step rate)
    stepper.set_timing(True, every=8)
    clocks = ClockSampler()
    if sample_clocks:
        clocks.start()
        time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    # step() ends by joining the observation stream (where one is used) into
    # the grid's stream before its counter update, so ev1 follows every launch
    stepper.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop() if sample_clocks else None
    ms = ev0.elapsed_time(ev1)
    kms, klaunch = stepper.kernel_time()
    in_use = sorted({g.kernel_in_use() for g in grids}, key=lambda kr: -kr[0])
    kname = " + ".join(KERNEL_NAMES[k] for k, _ in in_use)
    tiles = [[32 if k > 1 else None, r] for k, r in in_use]
    stepper.set_timing(False)
    stepper.sync()
    ms_max = rank_max(ms, dist)
    cells = sum(s.cells for s in specs)
    value = cells * steps * world / (ms_max * 1e-3) / 1e6

    # roofline of the step kernel(s): algorithmic bytes per launch / mean launch time
    peak, peak_kind = measured_peaks()
    bytes_step = sum(algorithmic_bytes(s, gc) for s, gc in zip(specs, gain_cells))
    # Two upper bounds of the step launches' mean duration: the launches
    # bracketed by CUDA events (every 8th step; the events cut the
    # programmatic overlap of those launches with the launch before them),
    # and the timed region per step (every launch of the step plus whatever
    # the observation adds).  With the observation on a second stream the step
    # launches run back to back and the second bound is the tighter one.
    ev_ms = kms / max(klaunch, 1)
    region_ms = ms_max / steps
    per_launch_ms = min(ev_ms, region_ms)
    launch_time_from = "per-launch CUDA events" if ev_ms <= region_ms else "timed region / steps"
    achieved = bytes_step / (per_launch_ms * 1e-3) / 1e9
    rec = {"value": round(value, 1), "ms_per_step": round(ms_max / steps, 5), "cells": cells,
           "launch_shape": ({"kernel": tune["kernel"], "by": tune["by"], "zdepth": tune["zdepth"],
                             "grid_blocks": tune["grid_blocks"], "order": ["costliest", "z"][tune["order"]],
                             "autotuned_over": tune["candidates"]}
                            if tune else "library default"),
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4), "traffic": None,
                        "kernel": kname, "tile": tiles[0] if len(tiles) == 1 else tiles,
                        "algorithmic_bytes_per_launch": bytes_step,
                        "mean_launch_ms": round(per_launch_ms, 5), "launch_time_from": launch_time_from,
                        "event_timed_launch_ms": round(ev_ms, 5), "peak_source": f"{peak_kind} hbm_gbs"},
           "launches": steps * (len(in_use) + 1) + 1,  # step kernel(s) and observation per step, one counter update
           "clocks": ck, "tune": tune, "n_kernels": len(in_use), "kname": kname, "tiles": tiles}
    return rec, grids, stepper


def recorded_traffic(args, workload, rec):
    """DRAM bytes of one step launch from the ncu captures of this workload in
    profiles/ (one record, or a list of them), when one was taken on the grid
    size, kernel and launch shape this run uses; else None."""
    prof = os.path.join(ROOT, "profiles", f"traffic_{workload}.json")
    if not os.path.exists(prof):
        return None
    with open(prof) as f:
        captures = json.load(f)
    if isinstance(captures, dict):
        captures = [captures]
    zd = rec["tune"]["zdepth"] if rec["tune"] else args.zdepth
    od = ["costliest", "z"][rec["tune"]["order"]] if rec["tune"] else (args.order or "costliest")
    for tr in captures:
        if rec["n_kernels"] == 1 and tr.get("kernel") == rec["kname"] and tr.get("tile") == rec["tiles"][0] \
                and tr.get("zdepth") == zd and tr.get("order", "costliest") == od and tr.get("cells") == rec["cells"]:
            return tr.get("dram_bytes_per_launch")
    return None


def run_gpu(args, rank, world, dist):
    import torch

    from paper_0802_3775_gb300 import build

    build.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    specs = workload_specs(args.workload, rank, args.steps + args.warmup)
    rec, grids, stepper = timed_workload(args, specs, world, dist, args.steps, args.warmup)
    roof = rec["roofline"]
    roof["traffic"] = recorded_traffic(args, args.workload, rec)

    batch_grids = []
    result = {
        "metric": METRIC, "value": rec["value"], "unit": "Mcell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if specs[0].precision == "f32" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload] + (f" -- reduced to {args.ncell}^3 unit cells "
                                                                 f"({specs[0].shape[0]}^3 grid)" if args.ncell else ""),
                   "grids_per_gpu": len(specs),
                   "cells_per_gpu": rec["cells"], "l2": "state larger than L2 (%.0f MB per GPU)" %
                   (rec["cells"] * (49 if specs[0].precision == "f32" else 97) / 1e6),
                   "parallelism": f"replicas x{world} (independent realizations)",
                   "launch": "direct launches; CUDA events around the step-kernel launch(es) of every 8th time step of the timed region",
                   "launch_shape": rec["launch_shape"]},
        "roofline": roof,
        "gpu_launches": rec["launches"],
        "clocks": rec["clocks"],
    }
    if rank == 0 and len(specs) > 1 and specs[0].precision == "f32":
        result.update(batch_extras(specs, grids, rec, args.steps))
    for g in grids:
        g.sync()
    if len(grids) > 1:
        stepper.close()
    for g in grids:
        g.close()

    # end to end through the public API with host inputs and host results
    result["e2e"] = run_e2e(args, specs, rank, dist)

    if rank == 0 and world == 1:
        if not args.no_serve:
            result["serve"] = serve_stream(count=args.serve_requests)
        if args.workload == "planewave" and not args.no_batch:
            result["batch"] = batch_record(args)
            result["gpu_launches"] += result["batch"]["gpu_launches"]
            result["lasing"] = lasing_record(args)
            result["gpu_launches"] += result["lasing"]["gpu_launches"]
        if not args.no_cpu:
            result["cpu_baseline"], result["oracle_error"] = cpu_leg(args)
    if rank == 0:
        print(json.dumps(result))


def batch_extras(specs, grids, rec, steps):
    """FP32 batched against the plain single-run FP64 GPU path: realizations
    per hour, and each of the first members against its FP64 GPU twin."""
    steps_run = 20000  # steps per realization of the batched workload
    rph32 = len(specs) / (rec["ms_per_step"] * 1e-3 * steps_run) * 3600.0
    rph64, nsamp = fp64_plain_rate(specs, steps_run)
    return {"vs_fp64_plain": {
        "fp32_batched_realizations_per_hour": round(rph32, 2),
        "fp64_plain_realizations_per_hour": round(rph64, 2), "factor": round(rph32 / rph64, 2),
        "steps_per_realization": steps_run,
        "note": f"FP64 path: each realization stepped alone (automatic kernel), mean of the first {nsamp}; "
                "both paths' errors against the FP64 oracle are in oracle_error"},
        "fp32_vs_fp64": fp32_vs_fp64_errors(specs, grids)}


def batch_record(args):
    """The 64-realization mixed batch (the batched workload) on this GPU,
    timed like the headline workload, with its FP64-plain comparison."""
    specs = workload_specs("batch", 0, args.steps + args.warmup)
    rec, grids, stepper = timed_workload(args, specs, 1, None, args.steps, args.warmup)
    out = {"workload": WORKLOAD_TEXT["batch"], "value": rec["value"], "unit": "Mcell-updates/s",
           "ms_per_step": rec["ms_per_step"], "realizations": len(specs), "cells": rec["cells"],
           "launch_shape": rec["launch_shape"], "roofline": rec["roofline"], "clocks": rec["clocks"],
           "gpu_launches": rec["launches"]}
    out.update(batch_extras(specs, grids, rec, args.steps))
    stepper.close()
    for g in grids:
        g.close()
    return out


def lasing_record(args):
    """The Maxwell-Bloch lasing workload (140^3, gain in the spheres) on this
    GPU, timed like the headline workload."""
    specs = workload_specs("lasing", 0, args.steps + args.warmup)
    rec, grids, _ = timed_workload(args, specs, 1, None, args.steps, args.warmup)
    for g in grids:
        g.close()
    rec["roofline"]["traffic"] = recorded_traffic(args, "lasing", rec)
    return {"workload": WORKLOAD_TEXT["lasing"], "value": rec["value"], "unit": "Mcell-updates/s",
            "ms_per_step": rec["ms_per_step"], "cells": rec["cells"], "launch_shape": rec["launch_shape"],
            "roofline": rec["roofline"], "clocks": rec["clocks"], "gpu_launches": rec["launches"]}


def run_e2e(args, specs, rank, dist):
    """Same metric through the public API: host sphere lists and parameters in,
    host probe / flux series out, all inside the timed region."""
    import torch

    from paper_0802_3775_gb300.fdtd import Grid

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    h2d = d2h = 0
    t0 = time.perf_counter()
    gs = []
    for s in specs:
        g = Grid.from_spec(s, record_capacity=args.steps + 16)
        configure_grid(args, g)
        h2d += s.spheres.nbytes if s.spheres is not None else 0
        gs.append(g)
    if len(gs) > 1:
        from paper_0802_3775_gb300.fdtd import Batch
        b = Batch(gs)
        configure_batch(args, b)
        b.set_graph(min(50, args.steps))
        b.step(args.steps)
        b.sync()
        b.close()
    else:
        gs[0].step(args.steps)
    for s, g in zip(specs, gs):
        fl = g.read_flux()
        pr = g.read_probes()
        d2h += fl.nbytes + pr.nbytes // (2 if s.precision == "f32" else 1)
        g.close()
    torch.cuda.synchronize()
    t = rank_max(time.perf_counter() - t0, dist)
    world = dist.get_world_size() if dist is not None else 1
    cells = sum(s.cells for s in specs)
    return {"value": round(cells * args.steps * world / t / 1e6, 1), "unit": "Mcell-updates/s",
            "h2d_bytes_per_step": round(h2d / args.steps, 1), "d2h_bytes_per_step": round(d2h / args.steps, 1),
            "includes": "grid creation from host sphere lists, device rasterization, set-up, steps "
                        "(CUDA-graph replays for batches), probe and flux series read back to the host"}


# ----------------------------------------------------------------------------- serving
def serve_stream(count: int = 32, rate_hz: float = 4.0, seed: int = 5000, capacity_mcell: float = None):
    """Served request stream with the served workload's sizes: Poisson
    arrivals at `rate_hz` of passive and lasing runs (grid edge 64..200 with
    the CPML, 5000..50000 steps), each submitted at its arrival time to one
    server (150 GB HBM budget, 64 slots, continuous batching at 500-step chunk
    boundaries).  Latency = completion - submission on the server's clock.
    The offered load rho = arrival rate x mean service time, the service
    time of a run being its cell-updates at the stream's measured throughput;
    rho > 1 means the queue grows over the stream, so latencies grow with its
    length."""
    from paper_0802_3775_gb300.serve import Server

    stream = inputs.request_stream(count, rate_hz=rate_hz, seed=seed, n_range=(64, 200), steps_range=(5000, 50000))
    work = [s.cells * s.steps for _, s in stream]
    srv = Server(hbm_budget_bytes=150 << 30, max_slots=64, steps_per_chunk=500)
    t0 = time.perf_counter()
    tickets = []
    for t_arr, spec in stream:
        now = time.perf_counter() - t0
        if t_arr > now:
            time.sleep(t_arr - now)
        tickets.append(srv.submit(spec, steps=spec.steps))
    lat, wait = [], []
    for t in tickets:
        r = srv.wait(t, timeout_s=1800.0)
        lat.append(r.done_s - r.submit_s)
        wait.append(r.admit_s - r.submit_s)
        srv.release(t)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    thr = sum(work) / wall / 1e6
    mean_service = (sum(work) / len(work)) / (thr * 1e6)
    lat.sort()
    return {"requests": count, "arrival_rate_hz": rate_hz,
            "offered_load": round(rate_hz * mean_service, 2),
            "p50_s": round(float(np.percentile(lat, 50)), 3), "p99_s": round(float(np.percentile(lat, 99)), 3),
            "max_s": round(lat[-1], 3), "mean_admission_wait_s": round(float(np.mean(wait)), 3),
            "realizations_per_hour": round(count / wall * 3600.0, 1),
            "mcell_updates_per_s": round(thr, 1), "failed": st["failed"],
            "stream": f"{count} requests, Poisson arrivals at {rate_hz}/s, passive and lasing runs of the served "
                      "workload generator, grid edge 64..200 incl. CPML, 5000..50000 steps, 150 GB budget, 64 slots, "
                      "500-step chunks; p50/p99 by linear interpolation between order statistics"}


def fp32_vs_fp64_errors(specs, grids, sample: int = 4):
    """Per realization (the first `sample` of the workload): the binary32
    member, as the batch left it, against the same realization stepped alone
    in binary64 on the GPU for as many steps: relative L2 of the six fields and
    of each flux series."""
    from paper_0802_3775_gb300.fdtd import Grid

    out = []
    for q, (s, g) in enumerate(zip(specs[:sample], grids[:sample])):
        n = int(g.steps_done)
        s64 = dataclasses.replace(s, precision="f64")
        g64 = Grid.from_spec(s64, record_capacity=n + 16)
        g64.step(n)
        g64.sync()
        F32, F64 = g.read_fields(), g64.read_fields()
        rec = {"realization": q, "gain": s.gain is not None, "steps": n,
               "fields_rel_l2": float(np.linalg.norm(F32 - F64) / max(np.linalg.norm(F64), 1e-300))}
        if g.nflux:
            T32, T64 = g.read_flux(), g64.read_flux()
            rec["flux_rel_l2"] = float(np.linalg.norm(T32 - T64) / max(np.linalg.norm(T64), 1e-300))
        out.append(rec)
        g64.close()
    return out


def fp64_plain_rate(specs, steps_run: int, steps: int = 60, sample: int = 4):
    """Realizations/hour of the plain single-run FP64 GPU path on the first
    `sample` realizations of the workload (each stepped alone, `steps` timed
    steps, extrapolated to `steps_run` steps per realization)."""
    import torch

    from paper_0802_3775_gb300.fdtd import Grid

    secs = []
    for s in specs[:sample]:
        s64 = dataclasses.replace(s, precision="f64")
        g = Grid.from_spec(s64, record_capacity=steps + 16)
        g.step(3)
        g.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(steps)
        g.sync()
        secs.append((time.perf_counter() - t0) / steps * steps_run)
        g.close()
    per = sum(secs) / len(secs)
    return 3600.0 / per, len(secs)


# ----------------------------------------------------------------------------- CPU oracle leg
# Everything below that runs the oracle is the benchmark's CPU leg: the oracle
# timed on the host cores, and the oracle results the GPU path is measured
# against.  Worker processes are started with "spawn" (never forked from a
# process that has touched the GPU).

def _single_thread_env():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def _oracle_timing_worker(spec, seconds, steps, warmup, barrier, queue, slot):
    """One process: build the oracle of `spec`, step `warmup` steps, wait for
    the others, then step for `steps` steps (or for `seconds` when steps is
    0); reports (slot, steps, seconds)."""
    _single_thread_env()
    sys.path.insert(0, ROOT)
    from oracle import Oracle
    o = Oracle.from_spec(spec)
    o.step(max(1, warmup))
    try:
        barrier.wait(timeout=600)
    except Exception:
        pass
    t0 = time.perf_counter()
    n = 0
    while True:
        o.step(1)
        n += 1
        t = time.perf_counter() - t0
        if (steps and n >= steps) or (not steps and t >= seconds):
            break
    queue.put((slot, n, t))


def oracle_processes(spec_cells, lasing):
    """Processes for the all-core oracle timing: one per allowed core, fewer
    when the host's available memory would not hold them at half of it
    (~360 B per cell for a passive oracle grid at its peak, ~600 with gain)."""
    cores = len(os.sched_getaffinity(0))
    avail = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    per = spec_cells * (600 if lasing else 360)
    if avail:
        cores = max(1, min(cores, int(0.5 * avail // per)))
    return cores


def time_oracle_all_cores(specs, seconds=10.0, steps=0, warmup=1):
    """Aggregate oracle rate with one process per spec stepping concurrently
    (independent realizations): sum over processes of cells x steps / time.
    Returns (Mcell/s, per-process (steps, seconds))."""
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(len(specs))
    queue = ctx.Queue()
    procs = [ctx.Process(target=_oracle_timing_worker, args=(s, seconds, steps, warmup, barrier, queue, q))
             for q, s in enumerate(specs)]
    for p in procs:
        p.start()
    res = [queue.get(timeout=1800) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    res.sort()
    rate = sum(specs[q].cells * n / t for q, n, t in res) / 1e6
    return rate, [(n, t) for _, n, t in res]


def _oracle_sample(spec, seconds: float):
    """Time the FP64 oracle on `spec` in this process for about `seconds`;
    returns (Mcell/s, steps, cells)."""
    from oracle import Oracle
    o = Oracle.from_spec(spec)
    o.step(1)
    t0 = time.perf_counter()
    n = 0
    while True:
        o.step(1)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    t = time.perf_counter() - t0
    return spec.cells * n / t / 1e6, n, spec.cells


def _oracle_run_worker(spec, steps, coef32):
    """Oracle results of `steps` steps of `spec` (fields, flux, probes)."""
    _single_thread_env()
    sys.path.insert(0, ROOT)
    from oracle import Oracle
    o = Oracle.from_spec(spec, coef32=coef32)
    o.step(steps)
    return (o.fields_memory_order(), o.flux_series() if o.fluxes else None,
            o.probe_series() if o.probes else None)


def _rel(a, b):
    nb = float(np.linalg.norm(np.asarray(b).ravel()))
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / (nb if nb > 0 else 1.0))


def oracle_errors(args, steps=150):
    """The GPU path against the FP64 oracle on reduced copies of the workload
    (2x2x2 unit cells of the same recipe; for the default workload also the
    first four members of the batch, reduced the same way and stepped as a
    batch): relative L2 of the six fields, of each flux series and of the
    probe series after `steps` steps, against the oracle fed the run's
    rounded coefficient tables (coef32 for binary32 runs) and, for the first
    run, the fields against the exact-coefficient oracle too.  The oracle
    runs go to a spawn pool while the GPU steps its copies."""
    import torch

    from paper_0802_3775_gb300.fdtd import Batch, Grid

    sets = [(args.workload, reduced_specs(args.workload, steps))]
    if args.workload == "planewave" and not args.no_batch:
        sets.append(("batch", reduced_specs("batch", steps)))
    runs = [(name, s) for name, specs in sets for s in specs]
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=min(len(runs) + 1, len(os.sched_getaffinity(0)))) as pool:
        rounded = [pool.apply_async(_oracle_run_worker, (s, steps, s.precision == "f32")) for _, s in runs]
        s0 = runs[0][1]
        exact = pool.apply_async(_oracle_run_worker, (s0, steps, False)) if s0.precision == "f32" else None
        gpu = []
        for name, specs in sets:
            grids = [Grid.from_spec(s, record_capacity=steps + 16) for s in specs]
            if len(grids) > 1:
                b = Batch(grids)
                b.step(steps)
                b.sync()
                b.close()
            else:
                grids[0].step(steps)
                grids[0].sync()
            for g in grids:
                gpu.append((g.read_fields(), g.read_flux() if g.nflux else None,
                            g.read_probes() if g.nprobe else None))
                g.close()
        torch.cuda.synchronize()
        ref = [p.get(timeout=1800) for p in rounded]
        ref_exact = exact.get(timeout=1800) if exact is not None else None
    out = []
    for q, ((name, s), (F, T, P), (Fo, To, Po)) in enumerate(zip(runs, gpu, ref)):
        rec = {"what": f"{name}: {s.shape[0]}x{s.shape[1]}x{s.shape[2]} "
                       f"{'lasing' if s.gain is not None else 'passive'} {s.precision}, {steps} steps",
               "fields_rel_l2": _rel(F, Fo)}
        if T is not None and To is not None:
            rec["flux_rel_l2"] = _rel(T, To)
        if P is not None and Po is not None:
            rec["probes_rel_l2"] = _rel(P, Po)
        if q == 0 and ref_exact is not None:
            rec["fields_rel_l2_vs_exact_coefficients"] = _rel(F, ref_exact[0])
        out.append(rec)
    return {"reference": "FP64 oracle fed the run's rounded coefficient tables", "runs": out}


def cpu_leg(args, seconds: float = 10.0):
    """The oracle on the host cores: all cores (one process per allowed core,
    each stepping its own realization of the workload) and one thread (one
    realization in this process); then the error checks against it."""
    specs = workload_specs(args.workload, 0, 1)
    spec = specs[1] if len(specs) > 1 and specs[1].gain is not None else specs[0]
    lasing = spec.gain is not None
    nproc = oracle_processes(spec.cells, lasing)
    if len(specs) == 1:
        pspecs = [workload_specs(args.workload, q, 1)[0] for q in range(nproc)]
    else:
        pspecs = [s for s in specs if (s.gain is not None) == lasing][:nproc]
    rate_all, per = time_oracle_all_cores(pspecs, seconds=seconds)
    v1, n1, _ = _oracle_sample(spec, seconds)
    sh = f"{spec.shape[0]}x{spec.shape[1]}x{spec.shape[2]}"
    baseline = {"value": round(rate_all, 3), "unit": "Mcell-updates/s", "cores": len(pspecs), "kind": "oracle",
                "sample": f"{len(pspecs)} processes, each stepping its own realization of the workload "
                          f"({'lasing' if lasing else 'passive'}, up to {sh} cells) for ~{seconds:.0f} s "
                          f"({min(n for n, _ in per)}..{max(n for n, _ in per)} steps); numpy FP64, one thread each",
                "single_thread": {"value": round(v1, 3), "cores": 1,
                                  "sample": f"{n1} steps of one {sh} realization of the workload (numpy FP64)"}}
    return baseline, oracle_errors(args)


def run_reference(args, rank):
    if rank != 0:
        return
    spec = workload_specs(args.workload, 0, 1)[0]
    budget = 150.0
    per_step = budget / max(1, args.steps + args.warmup)
    # shrink the sample grid until one oracle step fits the per-step budget
    sample = spec
    from oracle import Oracle
    probe = Oracle.from_spec(sample)
    t0 = time.perf_counter()
    probe.step(1)
    t1 = time.perf_counter() - t0
    note = "full realizations"
    shrink_ncell = None
    if t1 > per_step:
        shrink = max(0.2, (per_step / t1) ** (1 / 3))
        base = 6 if sample.gain is not None else 8
        shrink_ncell = max(2, int(round(base * shrink)))
    del probe

    def sample_spec(q):
        s = workload_specs(args.workload, q, 1)[0]
        if shrink_ncell is None:
            return s
        if s.gain is not None:
            return inputs.opal_lasing_f32(ncell=shrink_ncell, res=20, npml=10, sigma=0.05, pump=1e10, realization=q)
        return inputs.opal_planewave_f32(ncell=shrink_ncell, res=20, npml=12, sigma=0.06, realization=q,
                                         precision=s.precision)

    nproc = oracle_processes(sample_spec(0).cells, spec.gain is not None)
    pspecs = [sample_spec(q) for q in range(nproc)]
    if shrink_ncell is not None:
        s0 = pspecs[0]
        note = f"{shrink_ncell}^3 unit cells ({s0.shape[0]}^3 grid) of the same workload"
    # every process steps warmup + steps; the timed part is its last `steps`
    value, per = time_oracle_all_cores(pspecs, steps=args.steps, warmup=args.warmup)
    ms = 1e3 * statistics.mean(t / n for n, t in per)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "Mcell-updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload]},
        "cpu_baseline": {"value": round(value, 3), "unit": "Mcell-updates/s", "cores": nproc, "kind": "oracle",
                         "sample": note + f", numpy FP64 oracle, {nproc} processes (one per allowed core, each its "
                                          "own realization, one thread each)"},
        "e2e": {"value": round(value, 3), "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="planewave")
    ap.add_argument("--kernel", default="auto", choices=["auto", "plain", "tma", "pair"],
                    help="step kernel (default: the library's automatic choice)")
    ap.add_argument("--by", type=int, default=0, help="tile rows of the step kernel (0: library default)")
    ap.add_argument("--zdepth", type=int, default=0, help="planes per work item (0: library default)")
    ap.add_argument("--order", default="", choices=["", "costliest", "z"],
                    help="work-item order of the single-node kernels (default: the library's)")
    ap.add_argument("--no-serve", action="store_true", help="skip the served request stream")
    ap.add_argument("--serve-requests", type=int, default=32, help="requests of the served stream")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched sub-record of the default workload")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch shape")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle's CPU leg (timing and error checks)")
    ap.add_argument("--ncell", type=int, default=0,
                    help="unit cells per edge of the planewave / lasing workload (0: the workload's own; a smaller "
                         "grid for profiling captures)")
    args = ap.parse_args()
    if args.ncell:
        NCELL[args.workload] = args.ncell
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        td.init_process_group("nccl")
        dist = td
    run_gpu(args, rank, world, dist)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
