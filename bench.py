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

--impl reference times the FP64 CPU oracle (the reference of this build) on a
bounded sample of the same workload, on the host cores, rank 0 only.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
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
def workload_specs(name: str, rank: int, steps: int):
    """Run records of one rank's share of the workload."""
    if name == "planewave":
        # 8x8x8 unit cells at 20 cells/a + 12-cell CPML = 184^3, FP32, sigma 6 %
        return [inputs.opal_planewave_f32(ncell=8, res=20, npml=12, sigma=0.06, realization=rank, steps=steps)]
    if name == "lasing":
        # 6x6x6 unit cells at 20 cells/a + 10-cell CPML = 140^3, FP32 gain
        return [inputs.opal_lasing_f32(ncell=6, res=20, npml=10, sigma=0.05, pump=1e10, realization=rank,
                                       steps=steps)]
    if name == "dipole64":
        return [inputs.opal_dipole_f64(steps=steps)]
    if name == "batch":
        # 64 mixed-size realizations, half passive, half lasing (one launch per step)
        return inputs.mixed_batch(64, seed=4000 + 1000 * rank, steps=steps)
    if name == "planewave64":
        return [inputs.opal_planewave_f32(ncell=8, res=20, npml=12, sigma=0.06, realization=rank, steps=steps,
                                          precision="f64")]
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
    once and written once, material read once (see the design notes)."""
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
    if args.by or args.zdepth:
        g.set_launch(32, args.by, args.zdepth, 0)


def configure_batch(args, b):
    if args.kernel != "auto" or args.by or args.zdepth:
        b.set_launch(args.kernel, args.by, args.zdepth, 0)


def run_gpu(args, rank, world, dist):
    import torch

    from paper_0802_3775_gb300 import build
    from paper_0802_3775_gb300.fdtd import Grid

    build.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    specs = workload_specs(args.workload, rank, args.steps + args.warmup)
    cap = args.steps + args.warmup + 16
    grids = [Grid.from_spec(s, record_capacity=cap) for s in specs]
    for g in grids:
        configure_grid(args, g)
    gain_cells = []
    for g, s in zip(grids, specs):
        gain_cells.append(int(np.count_nonzero(g.get_material() & 64)) if s.gain is not None else 0)
    batch = None
    if len(grids) > 1:
        from paper_0802_3775_gb300.fdtd import Batch
        batch = Batch(grids)
        configure_batch(args, batch)
        stepper = batch
    else:
        stepper = grids[0]
    tune = None
    if not args.no_autotune and args.kernel == "auto" and not args.by and not args.zdepth:
        # launch shape picked by timing the candidates on this workload (state restored)
        tune = stepper.autotune(trial_steps=10 if batch is None else 4)
    stepper.step(args.warmup)
    stepper.sync()

    def barrier():
        if dist is not None:
            dist.barrier()

    # timed region: device events on the stream the kernels run on (torch's current stream)
    stream = torch.cuda.current_stream()
    # CUDA events around every 8th step-kernel launch of the timed region
    # (bracketing every launch costs a few per cent of the step rate)
    stepper.set_timing(True, every=8)
    clocks = ClockSampler()
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stepper.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    kernel = [stepper.kernel_time()]
    # step kernels in use (a batch launches one per kernel group each step)
    names = {1: "k_step", 2: "k_step_tma", 3: "k_step_pair"}
    in_use = sorted({g.kernel_in_use() for g in grids}, key=lambda kr: -kr[0])
    kind, rows = in_use[0]
    kname = " + ".join(names[k] for k, _ in in_use)
    tiles = [[32 if k > 1 else None, r] for k, r in in_use]
    stepper.set_timing(False)
    stepper.sync()
    ms_max = rank_max(ms, dist)
    cells = sum(s.cells for s in specs)
    value = cells * args.steps * world / (ms_max * 1e-3) / 1e6

    # roofline of the step kernel (dominant): algorithmic bytes per launch / mean launch time
    peak, peak_kind = measured_peaks()
    kms = sum(k[0] for k in kernel)
    klaunch = sum(k[1] for k in kernel)
    bytes_step = sum(algorithmic_bytes(s, gc) for s, gc in zip(specs, gain_cells))
    # Two upper bounds of the step launches' mean duration: the launches
    # bracketed by CUDA events (every 8th step; the events cut the
    # programmatic overlap of those launches with the launch before them),
    # and the timed region per step (every launch of the step plus whatever
    # the observation adds).  With the observation on a second stream the step
    # launches run back to back and the second bound is the tighter one.
    ev_ms = kms / max(klaunch, 1)
    region_ms = ms_max / args.steps
    per_launch_ms = min(ev_ms, region_ms)
    launch_time_from = "per-launch CUDA events" if ev_ms <= region_ms else "timed region / steps"
    achieved = bytes_step / (per_launch_ms * 1e-3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", f"traffic_{args.workload}.json")
    if os.path.exists(prof):
        with open(prof) as f:
            rec = json.load(f)
        # DRAM bytes of one launch from an ncu capture of this workload, when
        # it was taken on the kernel this run uses
        zd = tune["zdepth"] if tune else args.zdepth
        if len(in_use) == 1 and rec.get("kernel") == kname and rec.get("tile") == tiles[0] and rec.get("zdepth") == zd:
            traffic = rec.get("dram_bytes_per_launch")

    # end to end through the public API with host inputs and host results
    e2e = run_e2e(args, specs, rank, dist)

    launches = args.steps * (len(in_use) + 1) + 1  # step kernel(s) and observation per step, one counter update
    result = {
        "metric": METRIC, "value": round(value, 1), "unit": "Mcell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if specs[0].precision == "f32" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "grids_per_gpu": len(specs),
                   "cells_per_gpu": cells, "l2": "state larger than L2 (%.0f MB per GPU)" %
                   (sum(s.cells for s in specs) * (49 if specs[0].precision == "f32" else 97) / 1e6),
                   "parallelism": f"replicas x{world} (independent realizations)",
                   "launch": "direct launches; CUDA events around the step-kernel launch(es) of every 8th time step of the timed region",
                   "launch_shape": ({"kernel": tune["kernel"], "by": tune["by"], "zdepth": tune["zdepth"],
                                     "grid_blocks": tune["grid_blocks"], "autotuned_over": tune["candidates"]}
                                    if tune else "library default")},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": kname, "tile": tiles[0] if len(tiles) == 1 else tiles,
                     "algorithmic_bytes_per_launch": bytes_step,
                     "mean_launch_ms": round(per_launch_ms, 5), "launch_time_from": launch_time_from,
                     "event_timed_launch_ms": round(ev_ms, 5), "peak_source": f"{peak_kind} hbm_gbs"},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": ck,
    }
    if rank == 0:
        if world == 1 and not args.no_serve:
            result["serve"] = serve_stream(capacity_mcell=0.6 * value)
        if len(specs) > 1 and specs[0].precision == "f32":
            # FP32 batched vs plain single-run FP64 GPU path, realizations/hour
            steps_run = 20000  # steps per realization of the batched workload
            rph32 = len(specs) / (ms_max / args.steps * 1e-3 * steps_run) * 3600.0
            rph64, nsamp = fp64_plain_rate(specs, steps_run)
            result["vs_fp64_plain"] = {
                "fp32_batched_realizations_per_hour": round(rph32, 2),
                "fp64_plain_realizations_per_hour": round(rph64, 2), "factor": round(rph32 / rph64, 2),
                "steps_per_realization": steps_run,
                "note": f"FP64 path: each realization stepped alone (automatic kernel), mean of the first {nsamp}; "
                        "accuracy of both against the FP64 oracle is asserted by the parity tests"}
            result["fp32_vs_fp64"] = fp32_vs_fp64_errors(specs, grids)
        result["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(result))
    if batch is not None:
        batch.close()
    for g in grids:
        g.close()


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
def serve_stream(capacity_mcell: float, count: int = 48, load: float = 0.7, seed: int = 5000):
    """Served request stream (the served-workload generator scaled to run in
    about 15 s): Poisson arrivals of passive and lasing runs with grid edge
    64..160 (CPML included) and 2000..8000 steps, the arrival rate set so the
    offered load is `load` of `capacity_mcell`; every run is submitted at its
    arrival time to one server (150 GB budget, continuous batching).
    Latency = completion - submission, on the server's clock."""
    from paper_0802_3775_gb300.serve import Server

    stream = inputs.request_stream(count, rate_hz=1.0, seed=seed, n_range=(64, 160), steps_range=(2000, 8000))
    work = [s.cells * s.steps for _, s in stream]
    rate = load * capacity_mcell * 1e6 / (sum(work) / len(work))
    srv = Server(hbm_budget_bytes=150 << 30, max_slots=64, steps_per_chunk=500)
    t0 = time.perf_counter()
    tickets = []
    for t_arr, spec in stream:
        t_sub = t_arr / rate
        now = time.perf_counter() - t0
        if t_sub > now:
            time.sleep(t_sub - now)
        tickets.append(srv.submit(spec, steps=spec.steps))
    lat = []
    for t in tickets:
        r = srv.wait(t)
        lat.append(r.done_s - r.submit_s)
        srv.release(t)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat.sort()
    pick = lambda q: lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]
    return {"requests": count, "offered_load": load, "arrival_rate_hz": round(rate, 3),
            "p50_s": round(pick(0.50), 3), "p99_s": round(pick(0.99), 3), "max_s": round(lat[-1], 3),
            "realizations_per_hour": round(count / wall * 3600.0, 1),
            "mcell_updates_per_s": round(sum(work) / wall / 1e6, 1), "failed": st["failed"],
            "stream": "Poisson arrivals, grid edge 64..160 incl. CPML, 2000..8000 steps, half passive half "
                      "lasing (served-workload generator scaled down), 150 GB budget, 64 slots, 500-step chunks"}


def fp32_vs_fp64_errors(specs, grids, sample: int = 4):
    """Per realization (the first `sample` of the workload): the binary32
    member, as the batch left it, against the same realization stepped alone
    in binary64 on the GPU for as many steps: relative L2 of the six fields and
    of each flux series."""
    import numpy as np

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


# ----------------------------------------------------------------------------- CPU oracle
def _oracle_sample(spec, seconds: float):
    """Time the FP64 oracle on `spec` for about `seconds`; returns (Mcell/s, steps, cells)."""
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


def cpu_baseline(args, seconds: float = 12.0):
    specs = workload_specs(args.workload, 0, 1)
    spec = specs[1] if len(specs) > 1 and specs[1].gain is not None else specs[0]
    v, n, cells = _oracle_sample(spec, seconds)
    return {"value": round(v, 3), "unit": "Mcell-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} steps of one {spec.shape[0]}x{spec.shape[1]}x{spec.shape[2]} realization of the "
                      f"workload (numpy FP64, single thread)"}


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
    note = "full realization"
    if t1 > per_step:
        shrink = max(0.2, (per_step / t1) ** (1 / 3))
        if sample.gain is not None:
            ncell = max(2, int(round(6 * shrink)))
            sample = inputs.opal_lasing_f32(ncell=ncell, res=20, npml=10, sigma=0.05, pump=1e10)
        else:
            ncell = max(2, int(round(8 * shrink)))
            sample = inputs.opal_planewave_f32(ncell=ncell, res=20, npml=12, sigma=0.06,
                                               precision=spec.precision)
        note = f"{ncell}^3 unit cells ({sample.shape[0]}^3 grid) of the same workload"
        probe = Oracle.from_spec(sample)
    for _ in range(args.warmup):
        probe.step(1)
    t0 = time.perf_counter()
    probe.step(args.steps)
    t = time.perf_counter() - t0
    value = sample.cells * args.steps / t / 1e6
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "Mcell-updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload]},
        "cpu_baseline": {"value": round(value, 3), "unit": "Mcell-updates/s", "cores": 1, "kind": "oracle",
                         "sample": note + ", numpy FP64 oracle, single thread"},
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
    ap.add_argument("--no-serve", action="store_true", help="skip the served request stream")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch shape")
    args = ap.parse_args()
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
