"""Benchmark of the GB300 hydro stage: FP64 cell-updates/s on the production-shaped
workload (a stretched n = 1.5 polytrope passing a moving 1e3 Msun point mass with
excision; 2048 MeshBlocks of 32^3 = 67,108,864 cells, PPM + HLLC + SSP-RK2, Saha
H/He table with the learned-guess closure, dual energy).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One step = one synchronised RK2 step of every MeshBlock through the C ABI
(tde_step: CFL dt on the device, two stages, excision, resync).  Beside it: the
same mesh under LAT (effective rate, work fraction), and as extras the
entropy-wave workload (128^3), the EOS inversion, self-gravity, the remap and
LAT on other meshes.  Prints one JSON line (rank 0).  --impl reference times the
CPU oracle on the host cores instead, on a bounded sample of the workload.
Under torchrun each rank runs an independent replica on its own GPU (weak
scaling, no collective on the data path); the timed region is bracketed by a
barrier and the maximum over ranks is reported.
"""
import argparse
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

METRIC = "FP64 cell-updates/s and % of HBM roofline; surrogate+batched vs plain form at 1e-10"
UNIT = "cell-updates/s"
TABLE = os.path.join(ROOT, "paper_2609_37859_gb300", "data", "eos_saha_hhe_256.npz")
N, BLOCK, CFL = 128, 32, 0.3
RHO0, T0, MACH, AMP, SEED = 1e-8, 1e3, 1e7, 1e-3, 2609
SCHEME = dict(eos=1, dual=1, eta1=1e-3, eta2=1e-4, rho_floor=1e-20, p_floor=1e-20, u_floor=1e-20)
# algorithmic HBM bytes per cell-update (FP64, 6 conserved fields): stage 1 reads
# and writes 6 fields, stage 2 reads U0 and U1 and writes U2 -> 5 * 6 * 8
BYTES_PER_CELL_UPDATE = 240.0
WORKLOAD = ("entropy wave, 128^3 cells as 64 MeshBlocks of 32^3, ghost width 2, Saha H/He "
            "256x256 table, dual energy, PLM+HLLC+SSP-RK2, periodic, Mach 1e7, CFL 0.3")


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), \
        int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (the job time is the slowest rank's)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def whole_job_rate(units_per_rank, world, steps, ms):
    """Units processed by all ranks per second over the timed region."""
    return world * units_per_rank * steps / (ms * 1e-3)


def layout():
    from paper_2609_37859_gb300 import workloads as wl
    return wl.uniform_layout((N, N, N), (BLOCK, BLOCK, BLOCK), bc=(1, 1, 1), ng=2)


def eos_point(table_arrays):
    """P and c_s^2 of the background (rho0, T0) by bilinear table evaluation."""
    d = table_arrays
    lr = (np.log10(RHO0) - d["lrho"][0]) / ((d["lrho"][1] - d["lrho"][0]) / (d["n_rho"] - 1))
    lt = (np.log10(T0) - d["lT"][0]) / ((d["lT"][1] - d["lT"][0]) / (d["n_T"] - 1))
    i, j = int(lr), int(lt)
    w, s = lr - i, lt - j

    def bil(f):
        return (1 - w) * ((1 - s) * f[i, j] + s * f[i, j + 1]) + w * ((1 - s) * f[i + 1, j] + s * f[i + 1, j + 1])
    return 10 ** bil(d["log10_P"]), 10 ** bil(d["log10_cs2"])


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def barrier_fn(torch, dev, dist):
    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
    return barrier


def e2e_rotating(mesh, host_in, step_fn, torch, dev, stream):
    """End to end through the C ABI with host buffers: every step copies its
    state in from pinned host memory and its result back out.  Three device
    states rotate so that step k + 1's input copy and step k - 1's output copy
    (each on its own stream) overlap step k's kernels; the output copies go to
    one pinned buffer in stream order.  Returns run(n) and the bytes per copy."""
    host_out = torch.empty_like(host_in).pin_memory()
    U_main = mesh.U
    bufs = [U_main, torch.empty_like(U_main), torch.empty_like(U_main)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(3)]
    ev_done = [torch.cuda.Event() for _ in range(3)]
    ev_out = [torch.cuda.Event() for _ in range(3)]

    def run(n):
        with torch.cuda.stream(s_in):
            bufs[0].copy_(host_in, non_blocking=True)
            ev_in[0].record(s_in)
        for k in range(n):
            b, nx = k % 3, (k + 1) % 3
            if k + 1 < n:
                with torch.cuda.stream(s_in):
                    if k >= 2:
                        s_in.wait_event(ev_out[nx])   # that buffer's result is out
                    bufs[nx].copy_(host_in, non_blocking=True)
                    ev_in[nx].record(s_in)
            stream.wait_event(ev_in[b])
            mesh.bind(bufs[b])
            step_fn()
            ev_done[b].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done[b])
                host_out.copy_(bufs[b], non_blocking=True)
                ev_out[b].record(s_out)
        stream.wait_event(ev_out[(n - 1) % 3])

    def close():
        mesh.bind(U_main)
        bufs.clear()
    return run, close, host_in.numel() * 8


def sweep_roofline(prof, cells, flop_per_cell, slots_per_cell, traffic, fp64_peak, kernel_note):
    """roofline object of the dominant sweep: FP64 FLOP per cell (ncu SASS
    counters of that kernel on this workload) x cells per launch / its average
    CUDA-event launch time, against the FP64 FMA rate measured in this run.
    Counters of kernels that changed since their capture are passed as None:
    achieved and frac are then null."""
    sweeps = {k: prof[k] for k in ("sweep_x", "sweep_y", "sweep_z") if prof[k][0]}
    dom = max(sweeps, key=lambda k: sweeps[k][1])
    n_dom, ms_dom = sweeps[dom]
    avg_ms = ms_dom / max(n_dom, 1)
    roof = {"bound": "alu", "kernel": "k_sweep (%s)" % dom.replace("sweep_", ""),
            "unit": "TFLOP/s", "peak": fp64_peak * 1e-12,
            "peak_source": "FP64 FMA probe measured in this run (tde_probe_fp64)",
            "traffic": traffic.get(dom) if traffic else None,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read+write)",
            "avg_launch_ms": avg_ms, "launches": n_dom, "counters": kernel_note}
    fpc = flop_per_cell.get(dom) if flop_per_cell else None
    if fpc:
        ach = fpc * cells / (avg_ms * 1e-3)
        roof.update({"achieved": ach * 1e-12, "frac": ach / fp64_peak, "fp64_flop_per_cell": fpc})
        slots = slots_per_cell.get(dom) if slots_per_cell else None
        if slots:
            # the same kernel counted in FP64-pipe issue slots (peak = FMA rate / 2)
            rate = slots * cells / (avg_ms * 1e-3)
            roof["fp64_issue"] = {"slots_per_cell": slots, "achieved_slots_per_s": rate,
                                  "peak_slots_per_s": fp64_peak / 2, "frac": rate / (fp64_peak / 2)}
    else:
        roof.update({"achieved": None, "frac": None})
    return roof


def hbm_roofline(rate_per_gpu, peaks):
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    gbs = rate_per_gpu * BYTES_PER_CELL_UPDATE * 1e-9
    return {"bytes_per_cell_update": BYTES_PER_CELL_UPDATE, "achieved_gbs": gbs, "peak_gbs": hbm_peak,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs", "frac": gbs / hbm_peak}


def run_gpu(args):
    import torch
    from paper_2609_37859_gb300 import tde

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = tde.Context(local, stream)
    eos = tde.EOS.from_file(ctx, TABLE)
    barrier = barrier_fn(torch, dev, dist)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    # the learned closure of the headline needs the trained network (device
    # training: own forward / backward kernels and Adam, 2^20 table samples)
    train = eos.train(seed=SEED, n_samples=1 << 20, epochs=120, batch=4096, lr=3e-3)

    # ---- the headline: synchronised RK2 steps of the production-shaped mesh
    if args.no_headline:   # profiling runs of the other sections
        if rank == 0:
            line = {"metric": METRIC, "value": None, "unit": UNIT, "note": "headline skipped (--no-headline)"}
            fp64_peak = ctx.probe_fp64()
            if not args.no_eos:
                line["eos_inversion"] = eos_bench(ctx, eos, tde, torch, dev, args)
            if not args.no_grav:
                line["self_gravity"] = gravity_bench(ctx, tde, torch, dev, args)
            if not args.no_lat:
                line["lat_c4"] = lat_bench(ctx, eos, tde, torch, dev, args)
            if not args.no_c2:
                line["c2_entropy_wave"] = c2_section(ctx, eos, tde, torch, dev, args, fp64_peak, peaks)
            print(json.dumps(line), flush=True)
        return
    head = c5_headline(ctx, eos, tde, torch, dev, args, dist, world, barrier, stream)
    fp64_peak = ctx.probe_fp64()
    if rank == 0:
        steps = args.steps
        ms = head["ms"]
        value = whole_job_rate(head["cells"], world, steps, ms)
        e2e = whole_job_rate(head["cells"], world, steps, head["ms_e2e"])
        fresh = KERNELS_AS_CAPTURED_C5
        roof = sweep_roofline(head["prof"], head["cells"], FP64_FLOP_PER_CELL_C5 if fresh else None,
                              FP64_SLOTS_PER_CELL_C5 if fresh else None, DRAM_BYTES_C5 if fresh else None,
                              fp64_peak, C5_COUNTERS_NOTE)
        prof = head["prof"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": C5_WORKLOAD, "cells": head["cells"], "meshblocks": head["meshblocks"],
                       "global_batch": world * head["cells"],
                       "parallelism": "replica per GPU" if world > 1 else "1 GPU",
                       "step": "one synchronised SSP-RK2 step of every MeshBlock (tde_step: CFL dt on "
                               "the device, two stages with the learned closure, excision, resync)",
                       "l2": "working set %.1f GB per step > 129 MB L2 (no flush needed)" % head["state_gb"]},
            "hbm_roofline": hbm_roofline(value / world, peaks),
            "roofline": roof,
            "kernels_ms": {k: round(v[1], 4) for k, v in prof.items() if v[0]},
            "kernels_launches": {k: v[0] for k, v in prof.items() if v[0]},
            "gpu_launches": sum(v[0] for v in prof.values()),
            "clocks": head["clocks"],
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": head["copy_bytes"],
                    "d2h_bytes_per_step": head["copy_bytes"]},
            "counters": head["counts"],
            "autotune": head["autotune"],
            "lat": head["lat"],
            "training": {k: train[k] for k in ("samples", "epochs", "ms", "loss_first", "loss_last")},
        }
        if tuple(args.c5_grid) != (16, 16, 8):
            line["config"]["workload"] += "; profiling case: %d x %d x %d MeshBlocks around the star" % \
                tuple(args.c5_grid)
        torch.cuda.empty_cache()
        if not args.no_c2:
            line["c2_entropy_wave"] = c2_section(ctx, eos, tde, torch, dev, args, fp64_peak, peaks)
            torch.cuda.empty_cache()
        if not args.no_eos:
            line["eos_inversion"] = eos_bench(ctx, eos, tde, torch, dev, args)
        if not args.no_grav:
            line["self_gravity"] = gravity_bench(ctx, tde, torch, dev, args)
        if not args.no_remap:
            line["remap"] = remap_bench(ctx, tde, torch, dev, args, n=args.remap_n)
        if not args.no_smr:
            line["lat_refined"] = smr_bench(ctx, tde, torch, dev, args)
        if not args.no_lat:
            line["lat_c4"] = lat_bench(ctx, eos, tde, torch, dev, args)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def c2_section(ctx, eos, tde, torch, dev, args, fp64_peak, peaks):
    """The entropy-wave workload (C2: 128^3 as 64 x 32^3, PLM, Saha table in cgs,
    dual energy, Mach 1e7): device rate, end to end, roofline of its dominant
    sweep, conservation audit and the closure modes."""
    from paper_2609_37859_gb300 import workloads as wl
    tab = np.load(TABLE)
    Pw, cs2 = eos_point(tab)
    lay = layout()
    W, _ = wl.entropy_wave(lay, RHO0, Pw, MACH * np.sqrt(cs2), amp=AMP, seed=SEED)
    mesh = tde.Mesh(ctx, lay, tde.make_params(**SCHEME), eos)
    mesh.prim_to_cons(torch.from_numpy(np.ascontiguousarray(W)).to(dev))
    U_init = mesh.U.clone()
    ncell = lay.ncells
    tiles, tile_ms = mesh.autotune(reps=3)
    steps = max(args.steps, 20)
    for _ in range(args.warmup):
        mesh.step(cfl=CFL)
    torch.cuda.synchronize(dev)
    flat_int = torch.from_numpy(lay.interior_flat()).to(dev)

    def audit():
        G = mesh.U[:5][:, flat_int].cpu().numpy()
        return [math.fsum(G[q]) for q in range(5)], [math.fsum(np.abs(G[q])) for q in range(5)]
    sums0, scale0 = audit()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    torch.cuda.nvtx.range_push("c2_timed_steps")   # lets a profiler select these launches
    e0.record(stream)
    for _ in range(steps):
        mesh.step(cfl=CFL)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile_read()
    ctx.profile(False)
    sums1, _ = audit()
    conservation = {"steps": steps, "summation": "math.fsum (correctly rounded) over the interior cells",
                    "rel_drift": {name: abs(sums1[q] - sums0[q]) / max(scale0[q], 1e-300)
                                  for q, name in enumerate(("mass", "momentum_x", "momentum_y", "momentum_z",
                                                            "total_energy"))}}
    del flat_int
    host_in = U_init.cpu().pin_memory()
    mesh.set_time(0.0)
    run, close, nbytes = e2e_rotating(mesh, host_in, lambda: mesh.step(cfl=CFL), torch, dev, stream)
    run(max(1, args.warmup))
    torch.cuda.synchronize(dev)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    run(steps)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    ms_e2e = f0.elapsed_time(f1)
    close()
    value = ncell * steps / (ms * 1e-3)
    out = {"workload": WORKLOAD, "cells": ncell, "steps": steps, "ms_per_step": ms / steps,
           "value": value, "unit": UNIT,
           "e2e": {"value": ncell * steps / (ms_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                   "d2h_bytes_per_step": nbytes},
           "hbm_roofline": hbm_roofline(value, peaks),
           "roofline": sweep_roofline(prof, ncell, FP64_FLOP_PER_CELL_SWEEP if KERNELS_AS_CAPTURED else None,
                                      FP64_SLOTS_PER_CELL_SWEEP if KERNELS_AS_CAPTURED else None,
                                      DRAM_BYTES_SWEEP if KERNELS_AS_CAPTURED else None, fp64_peak,
                                      "profiles/k_sweep_c2_entropy_wave_ncu.md"),
           "kernels_ms": {k: round(v[1], 4) for k, v in prof.items() if v[0]},
           "autotune": autotune_report(tiles, tile_ms),
           "counters": mesh.counts(),
           "conservation": conservation}
    if not args.no_eos:
        out["closure_modes"] = closure_bench(mesh, U_init, tde, torch, dev, args)
    del mesh, U_init, host_in
    return out


# FP64 operations (DADD + DMUL + 2 x DFMA thread-instructions, ncu SASS counters)
# per interior cell in one launch of each sweep kernel on this workload, and the
# DRAM bytes of one launch; profiles/k_sweep_c2_entropy_wave_ncu.md holds the
# capture.  They describe the kernels as captured: set KERNELS_AS_CAPTURED to
# False (achieved, frac and traffic reported as null) whenever a sweep kernel
# changes.
FP64_FLOP_PER_CELL_SWEEP = {"sweep_x": 205.2, "sweep_y": 169.7, "sweep_z": 295.7}
DRAM_BYTES_SWEEP = {"sweep_x": 268.5e6, "sweep_y": 402.6e6, "sweep_z": 545.1e6}
# FP64-pipe issue slots (warp instructions x 32) per interior cell: a DADD or DMUL
# holds the pipe as long as a DFMA, so the pipe's busy fraction is slots / peak.
FP64_SLOTS_PER_CELL_SWEEP = {"sweep_x": 187.3, "sweep_y": 187.3, "sweep_z": 275.3}
KERNELS_AS_CAPTURED = True
# The same for the headline's sweeps (production-shaped mesh, PPM, point mass),
# from ncu on the 8 x 8 x 4 MeshBlocks around the star of that mesh (8.4 M
# cells, the same cells and scheme; the full mesh holds ~36 GB on the device,
# too much for a multi-pass capture), two launches of each sweep averaged,
# DRAM bytes scaled to the full mesh by its cells (x 8); a one-pass capture of
# the full mesh gives the same FP64 slots per cell within 2 %.
FP64_FLOP_PER_CELL_C5 = {"sweep_x": 240.7, "sweep_y": 224.8, "sweep_z": 355.3}
FP64_SLOTS_PER_CELL_C5 = {"sweep_x": 185.5, "sweep_y": 174.9, "sweep_z": 268.0}
DRAM_BYTES_C5 = {"sweep_x": 11.00e9, "sweep_y": 15.48e9, "sweep_z": 21.29e9}
KERNELS_AS_CAPTURED_C5 = True
C5_COUNTERS_NOTE = "profiles/k_sweep_c5_production_ncu.md (8x8x4-block case of the same mesh)"


SHAPE_NAMES = ("8 lanes x 288 threads", "16 lanes x 288 threads", "4 lanes x 160 threads")


def autotune_report(tiles, ms):
    return {"chosen": {d: SHAPE_NAMES[t] for d, t in zip("xyz", tiles)},
            "launch_ms": {d: {SHAPE_NAMES[k]: (round(v, 4) if v >= 0 else None) for k, v in enumerate(row)}
                          for d, row in zip("xyz", ms)}}


def closure_bench(mesh, U_init, tde, torch, dev, args):
    """The bench step with each way of inverting the table in cons -> prim
    (same results, checked bitwise): FP32-guided bisection (the headline), plain
    FP64 bisection, and the learned guess + one FP64 Newton step."""
    out, ref = {}, None
    nsteps = 10
    for name, mode in (("bisect_fp32_guided", tde.INVERT_BISECT), ("bisect_plain", tde.INVERT_BISECT_PLAIN),
                       ("surrogate_newton", tde.INVERT_SURROGATE)):
        mesh.set_params(tde.make_params(eos_mode=mode, **SCHEME))
        mesh.U.copy_(U_init)
        mesh.set_time(0.0)
        for _ in range(max(1, args.warmup)):
            mesh.step(cfl=CFL)
        mesh.U.copy_(U_init)
        mesh.set_time(0.0)
        mesh.counts(reset=True)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(nsteps):
            mesh.step(cfl=CFL)
        b.record()
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / nsteps
        c = mesh.counts()
        U = mesh.U.clone()
        if ref is None:
            ref = U
        out[name] = {"ms_per_step": ms, "cell_updates_per_s": mesh.layout.ncells / (ms * 1e-3),
                     "identical_to_fp32_guided": bool(torch.equal(U, ref)),
                     "accepted_fraction": c["surrogate_accepted"] / (mesh.layout.ncells * 2 * nsteps)}
    # the Riemann solver of the paper's production runs (HLLE) against HLLC
    for name, rs in (("hllc", tde.RIEMANN_HLLC), ("hlle", tde.RIEMANN_HLLE)):
        mesh.set_params(tde.make_params(riemann=rs, **SCHEME))
        mesh.U.copy_(U_init)
        mesh.set_time(0.0)
        mesh.step(cfl=CFL)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(nsteps):
            mesh.step(cfl=CFL)
        b.record()
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / nsteps
        out["riemann_" + name] = {"ms_per_step": ms, "cell_updates_per_s": mesh.layout.ncells / (ms * 1e-3)}
    mesh.set_params(tde.make_params(**SCHEME))
    return {"workload": "the bench step (C2), %d steps per mode" % nsteps, **out}


# ------------------------------------------------------- EOS inversion (C3) ---

EOS_CELLS = 1 << 24


def eos_bench(ctx, eos, tde, torch, dev, args):
    """2^24 (rho, e) cells -> (T, P, cs2): table bisection against the learned guess
    plus one Newton step (identical results, checked), with the network trained on
    the device at the start of the run (2^20 table samples)."""
    from paper_2609_37859_gb300 import workloads as wl
    g = torch.Generator(device=dev)
    g.manual_seed(SEED)
    rho, T0 = wl.c3_inputs(EOS_CELLS, g, dev)
    e = torch.empty_like(rho)
    eos.eval_rhoT(rho, T0, e=e)
    del T0
    res = {}
    outs = {}
    for name, mode in (("bisect_plain", tde.INVERT_BISECT_PLAIN), ("bisect", tde.INVERT_BISECT),
                       ("surrogate", tde.INVERT_SURROGATE)):
        T, P, c2 = (torch.empty_like(rho) for _ in range(3))
        for _ in range(2):
            eos.invert(rho, e, T=T, P=P, cs2=c2, mode=mode)
        before = eos.counts()["surrogate_accepted"]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        torch.cuda.synchronize(dev)
        e0.record()
        for _ in range(reps):
            eos.invert(rho, e, T=T, P=P, cs2=c2, mode=mode)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        acc = (eos.counts()["surrogate_accepted"] - before) / (reps * EOS_CELLS)
        res[name] = {"cells_per_s": EOS_CELLS / (ms * 1e-3), "ms": ms, "accepted": acc,
                     "hbm_gbs": EOS_CELLS * 40 / (ms * 1e-3) * 1e-9}
        outs[name] = (T, P, c2)
    same = all(torch.equal(a, b) and torch.equal(a, c)
               for a, b, c in zip(outs["bisect"], outs["surrogate"], outs["bisect_plain"]))
    return {"workload": "2^24 cells, log10 rho U[-14, 2], log10 T uniform in the recombination band "
                        "(1 % H+ to 99 % He2+ at that density, Saha) mapped to e by the table; "
                        "outputs T, P, cs2 (40 B/cell)",
            "bisect_plain": res["bisect_plain"], "bisect_fp32_guided": res["bisect"],
            "surrogate_newton": res["surrogate"],
            "speedup_vs_plain": res["bisect_plain"]["ms"] / res["surrogate"]["ms"],
            "speedup_vs_fp32_guided": res["bisect"]["ms"] / res["surrogate"]["ms"],
            "identical_results": bool(same)}


# ------------------------------------------------------------- LAT stream (C4) ---

def lat_bench(ctx, eos, tde, torch, dev, args):
    """The LAT workload: 384 x 32^3 + 128 x 16^3 MeshBlocks (13.1 M cells), PPM,
    Saha table in code units, dual energy, point mass with excision, N_LAT = 5.
    Compares, over the same physical time f_max dt0: LAT windows (per-level
    batched launches, replayed as a CUDA graph), synchronised steps of dt0 (every
    block every fine step), and the plain form of one launch sequence per block
    and stage (measured on one step)."""
    from paper_2609_37859_gb300 import workloads as wl
    lay, f, bhp = wl.stream_c4()
    rho_cgs = torch.from_numpy(np.ascontiguousarray(f["rho"] * wl.RHO0_CGS).ravel()).to(dev)
    Tt = torch.from_numpy(np.ascontiguousarray(f["T"]).ravel()).to(dev)
    Pc = torch.empty_like(rho_cgs)
    eos.eval_rhoT(rho_cgs, Tt, P=Pc)
    P_code = (Pc / (wl.RHO0_CGS * wl.V0_CGS ** 2)).cpu().numpy().reshape(f["rho"].shape)
    del rho_cgs, Tt, Pc
    W = wl.prim_state(lay, f["rho"], f["vx"], f["vy"], f["vz"], P_code)
    params = tde.make_params(eos=tde.EOS_TABLE, recon=tde.RECON_PPM, dual=1, eta1=1e-3, eta2=1e-4,
                             rho_floor=1e-17, p_floor=1e-30, u_floor=1.5e-30,
                             unit_rho=wl.RHO0_CGS, unit_e=wl.V0_CGS ** 2)
    mesh = tde.Mesh(ctx, lay, params, eos)
    mesh.prim_to_cons(torch.from_numpy(np.ascontiguousarray(W)).to(dev))
    del W
    bh = tde.make_bh(on=1, excise=1, GM=bhp["GM"], r_soft=bhp["r_soft"], r_exc=bhp["r_exc"],
                     x0=bhp["x0"])
    U0 = mesh.U.clone()
    n_lat = 5
    fac, dt0, fmax = mesh.lat_assign(n_lat, CFL, merge_frac=0.01, bh=bh)
    cells = np.array([b[3] * b[4] * b[5] for b in lay.blocks], dtype=np.float64)
    work = float((cells * (fmax // fac)).sum() / (cells.sum() * fmax))
    levels = {int(k): int((fac == k).sum()) for k in np.unique(fac)}

    def timed(fn, reps):
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    def set_mode(mode):
        mesh.set_params(tde.make_params(eos_mode=mode, **{f: getattr(params, f) for f, _ in params._fields_
                                                          if f != "eos_mode"}))

    def lat_arm(mode):
        set_mode(mode)
        mesh.U.copy_(U0)
        mesh.set_time(0.0)
        mesh.lat_set_factors(fac, dt0)
        mesh.lat_window(bh=bh, use_graph=False)   # warm-up: eager, then capture
        mesh.lat_window(bh=bh, use_graph=True)
        mesh.U.copy_(U0)
        mesh.set_time(0.0)
        mesh.lat_window(bh=bh, use_graph=True)
        U1w = mesh.U.clone()
        mesh.U.copy_(U0)
        mesh.set_time(0.0)
        mesh.counts(reset=True)
        ms = timed(lambda: mesh.lat_window(bh=bh, use_graph=True), 2)
        c = mesh.counts(reset=True)
        c["surrogate_accepted"] //= 2   # per window
        return ms, U1w, c

    # LAT with tiles autotuned on this mesh: FP32-guided bisection (the GB300
    # form) and the learned guess (the learned + batched form)
    tiles, tile_ms = mesh.autotune(bh=bh, reps=2)
    ms_lat, U_lat, lat_counts = lat_arm(tde.INVERT_BISECT)
    ms_lat_sur, U_sur, sur_counts = lat_arm(tde.INVERT_SURROGATE)
    same_lat = bool(torch.equal(U_lat, U_sur))
    del U_sur
    # the same windows with one persistent launch per level sub-step
    set_mode(tde.INVERT_BISECT)
    assert mesh.set_lat_mode(tde.LAT_PERSISTENT)
    ms_lat_pers, U_pers, pers_counts = lat_arm(tde.INVERT_BISECT)
    same_pers = bool(torch.equal(U_lat, U_pers)) and pers_counts == lat_counts
    mesh.set_lat_mode(tde.LAT_SEQUENCE)
    del U_pers
    set_mode(tde.INVERT_BISECT)
    # synchronised steps of dt0 over the same physical time
    mesh.U.copy_(U0)
    mesh.set_time(0.0)
    mesh.step(dt=dt0, bh=bh)
    mesh.U.copy_(U0)
    mesh.set_time(0.0)

    def sync_window():
        for _ in range(fmax):
            mesh.step(dt=dt0, bh=bh)
    ms_sync = timed(sync_window, 1)
    flat = torch.from_numpy(lay.interior_flat()).to(dev)
    vs_sync = lat_vs_sync_metrics(torch, U_lat[0][flat], mesh.U[0][flat], params.rho_floor)
    del U_lat, flat
    # plain form: plain FP64 table bisection, the default tile shape, one launch
    # sequence per block and stage; one step of dt0
    set_mode(tde.INVERT_BISECT_PLAIN)
    mesh.set_tiles((0, 0, 0))
    ids = torch.arange(lay.nb, dtype=torch.int32, device=dev)
    dtb = torch.full((lay.nb,), dt0, dtype=torch.float64, device=dev)
    tb = torch.zeros(lay.nb, dtype=torch.float64, device=dev)
    mesh.U.copy_(U0)

    def plain_step():
        for st in (0, 1):
            for b in range(lay.nb):
                mesh.hydro_stage(st, dtb, tb, ids=ids[b:b + 1], bh=bh)
    plain_step()
    ms_plain_step = timed(plain_step, 1)
    set_mode(tde.INVERT_BISECT)
    ncell = lay.ncells
    upd = ncell * fmax
    del mesh, U0
    torch.cuda.empty_cache()
    return {"workload": "cold stream on an ellipse (r_p 10, r_a 28 Rsun) around 1e3 Msun with excision, "
                        "384 x 32^3 + 128 x 16^3 MeshBlocks, PPM+HLLC, Saha table, dual energy, N_LAT 5",
            "cells": ncell, "meshblocks": lay.nb, "f_max": int(fmax), "blocks_per_factor": levels,
            "work_fraction": work, "work_reduction": 1.0 - work,
            "autotune": autotune_report(tiles, tile_ms),
            "lat_window_ms": ms_lat, "sync_window_ms": ms_sync,
            "persistent_level_window_ms": ms_lat_pers,
            "persistent_level_identical_to_lat": same_pers,
            "learned_batched_window_ms": ms_lat_sur,
            "learned_batched_identical_to_lat": same_lat,
            "learned_accepted_per_window": sur_counts["surrogate_accepted"],
            "closure_interior_cell_stages_per_window": lat_counts_cells(lay, fac, fmax),
            "plain_per_block_step_ms": ms_plain_step, "plain_window_ms_est": ms_plain_step * fmax,
            "lat_speedup_vs_sync": ms_sync / ms_lat,
            "lat_vs_sync_one_window": vs_sync,
            "lat_speedup_vs_plain": ms_plain_step * fmax / ms_lat,
            "learned_batched_speedup_vs_plain": ms_plain_step * fmax / ms_lat_sur,
            "effective_cell_updates_per_s": {"lat": upd / (ms_lat * 1e-3), "sync": upd / (ms_sync * 1e-3),
                                             "learned_batched": upd / (ms_lat_sur * 1e-3),
                                             "plain": ncell / (ms_plain_step * 1e-3)},
            "plain_form": "plain FP64 table bisection, default tiles, one launch sequence per block and stage",
            "learned_batched_form": "learned guess + one FP64 Newton step, autotuned tiles, per-level batched "
                                    "launches replayed as a CUDA graph",
            "lat_counters": lat_counts}


def lat_vs_sync_metrics(torch, rho_lat, rho_sync, rho_floor):
    """The LAT-vs-synchronised comparison of Sec. 7.4 over the interior cells (the
    sample points): norms of the relative density difference (rho_LAT - rho_sync) /
    rho_sync (Eq. lat-density-error-norms), the Pearson coefficient of log10 rho
    and the Jaccard overlap of the cells denser than 100 rho_floor."""
    d = (rho_lat - rho_sync) / rho_sync
    q1, q2 = torch.log10(rho_lat), torch.log10(rho_sync)
    a, b = q1 - q1.mean(), q2 - q2.mean()
    c = (a * b).sum() / torch.sqrt((a * a).sum() * (b * b).sum())
    d1, d2 = rho_lat > 1e2 * rho_floor, rho_sync > 1e2 * rho_floor
    union = int((d1 | d2).sum())
    return {"L1": float(d.abs().mean()), "L2": float(torch.sqrt((d * d).mean())),
            "Linf": float(d.abs().max()), "C_logrho": float(c),
            "J_dense": int((d1 & d2).sum()) / max(union, 1),
            "paper_context": "production restart, 7 levels, f_max 128, 5 code times: L1/L2/Linf = "
                             "9.04e-3 / 2.94e-2 / 1.64e-1, C_logrho 0.99975, J_dense 1"}


def lat_counts_cells(lay, fac, fmax):
    """Interior cell-stages of one LAT window (2 stages per update; slow blocks
    also convert their ghost cells, which this count leaves out)."""
    cells = np.array([b[3] * b[4] * b[5] for b in lay.blocks], dtype=np.int64)
    return int((cells * (fmax // fac)).sum() * 2)


# ------------------------------------------------------------ self-gravity ---

def gravity_bench(ctx, tde, torch, dev, args, n=256):
    """Self-gravity multigrid on an n^3 periodic grid (n^3 / 32^3 MeshBlocks):
    time per V-cycle as the paper measures it (runs of 6 and 2 fixed V-cycles,
    difference / 4), V-cycles and time to a 1e-9 rms defect from zero and from the
    previous potential, and the fine-level traffic of a V-cycle against HBM."""
    from paper_2609_37859_gb300 import workloads as wl
    lay = wl.uniform_layout((n, n, n), (32, 32, 32), bc=(1, 1, 1), ng=2)
    W = wl.random_smooth(lay, seed=SEED, drho=0.5, P0=1.0, modes=4)
    mesh = tde.Mesh(ctx, lay, tde.make_params())
    mesh.prim_to_cons(torch.from_numpy(np.ascontiguousarray(W)).to(dev))
    del W
    G = 1.0 / (4.0 * np.pi)
    mesh.gravity_solve(G, 0.0, tol=0.0, max_cycles=2, warm=False)   # allocation, warm-up

    def timed(fn):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize(dev)
        return (time.perf_counter() - t0) * 1e3, r
    ms6, _ = timed(lambda: mesh.gravity_solve(G, 0.0, tol=0.0, max_cycles=6, warm=False))
    ms2, _ = timed(lambda: mesh.gravity_solve(G, 0.0, tol=0.0, max_cycles=2, warm=False))
    per_cycle = (ms6 - ms2) / 4.0
    ms_cold, (ncold, dcold) = timed(lambda: mesh.gravity_solve(G, 0.0, tol=1e-9, max_cycles=30, warm=False))
    # a warm start after a small change of the density (one hydro step)
    mesh.step(cfl=CFL)
    ms_warm, (nwarm, dwarm) = timed(lambda: mesh.gravity_solve(G, 0.0, tol=1e-9, max_cycles=30, warm=True))
    ncell = lay.ncells
    # fine-level algorithmic traffic per V-cycle: 5 red-black sweeps (2 pre, 2 post,
    # 1 extra) of 24 B/cell (phi and source read, phi written), restriction 19,
    # prolongation 18, the defect norm 16 B/cell; coarser levels add 1/7
    bytes_cycle = ncell * (5 * 24 + 19 + 18 + 16) * 8.0 / 7.0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    # the full-multigrid start (the paper's start for a first or remapped solve)
    ms_fmg, (nfmg, dfmg) = timed(lambda: mesh.gravity_solve(G, 0.0, tol=1e-9, max_cycles=30, warm=False, fmg=True))
    del mesh
    torch.cuda.empty_cache()
    # isolated boundaries (multipole, l_max = 4): a centrally condensed cloud on
    # an outflow mesh, from the full-multigrid start
    lay_i = wl.uniform_layout((n, n, n), (32, 32, 32), domain=((-1, 1),) * 3, bc=(0, 0, 0), ng=2)
    xi, yi, zi = lay_i.cell_centres()
    rho_i = 1e-4 + np.exp(-((xi - 0.1) ** 2 + yi ** 2 + (zi + 0.05) ** 2) / (2 * 0.2 ** 2))
    Wi = wl.prim_state(lay_i, rho_i, 0.0, 0.0, 0.0, 0.1 * rho_i)
    del xi, yi, zi, rho_i
    mesh = tde.Mesh(ctx, lay_i, tde.make_params())
    mesh.prim_to_cons(torch.from_numpy(np.ascontiguousarray(Wi)).to(dev))
    del Wi
    mesh.gravity_solve(G, 0.0, tol=0.0, max_cycles=2, warm=False, isolated=True, fmg=True)   # warm-up
    ms6i, _ = timed(lambda: mesh.gravity_solve(G, 0.0, tol=0.0, max_cycles=6, warm=True, isolated=True))
    ms2i, _ = timed(lambda: mesh.gravity_solve(G, 0.0, tol=0.0, max_cycles=2, warm=True, isolated=True))
    ms_iso, (niso, diso) = timed(lambda: mesh.gravity_solve(G, 0.0, tol=1e-9, max_cycles=30, warm=False,
                                                            isolated=True, lmax=4, fmg=True))
    del mesh
    torch.cuda.empty_cache()
    return {"workload": "%d^3 periodic, %d MeshBlocks of 32^3, random smooth density, G = 1/(4 pi)" %
                        (n, lay.nb),
            "ms_per_vcycle": per_cycle, "cold": {"vcycles": ncold, "defect": dcold, "ms": ms_cold},
            "fmg_start": {"vcycles_after": nfmg, "defect": dfmg, "ms": ms_fmg},
            "isolated": {"workload": "%d^3 on [-1, 1]^3, outflow mesh, Gaussian cloud (sigma 0.2) over a "
                                     "1e-4 floor, multipole boundary values to l_max = 4" % n,
                         "ms_per_vcycle": (ms6i - ms2i) / 4.0,
                         "fmg_solve": {"vcycles_after": niso, "defect": diso, "ms": ms_iso}},
            "warm_after_one_step": {"vcycles": nwarm, "defect": dwarm, "ms": ms_warm},
            "hbm": {"algorithmic_bytes_per_vcycle": bytes_cycle,
                    "achieved_gbs": bytes_cycle / (per_cycle * 1e-3) * 1e-9, "peak_gbs": hbm,
                    "frac": bytes_cycle / (per_cycle * 1e-3) * 1e-9 / hbm},
            "paper_context": "Table mg-cost: 6.2 / 11.3 ms per V-cycle (16^3 / 32^3 MeshBlocks, 5 AMR "
                             "levels, two V100s; AthenaK public solver 22.4 / 49.6 ms)"}


def smr_bench(ctx, tde, torch, dev, args):
    """LAT across coarse-fine interfaces (Sec. 7.1): a blast wave (ideal gas,
    PLM + HLLE, dual energy) at the centre of a statically refined mesh, the
    level-0 grid 128^3 in 16^3 MeshBlocks, refined twice (levels 1 and 2, 2:1
    balanced) within r = 0.15 of the centre: 1912 blocks, 7.8 M cells.  Over the
    same physical time f_max dt0: one LAT window (CUDA graph) against f_max
    synchronised steps of dt0 (each one window with every factor 1), and the
    density difference between the two (the paper's blast-wave comparison)."""
    from paper_2609_37859_gb300 import workloads as wl

    def sphere(lo, hi, L):
        return sum(max(lo[a], 0.0, -hi[a]) ** 2 for a in range(3)) < 0.15 ** 2

    lay = wl.smr_layout((128, 128, 128), (16, 16, 16), ((-0.5, 0.5),) * 3, (0, 0, 0), 2, sphere, 2)
    x, y, z, _ = lay.interior_centres()
    r2 = x * x + y * y + z * z
    W = wl.prim_cells(lay, 1.0, 0.0, 0.0, 0.0, np.where(r2 < 0.04 ** 2, 10.0, 1e-2))
    params = tde.make_params(dual=1, eta1=1e-3, eta2=1e-4, riemann=tde.RIEMANN_HLLE)
    mesh = tde.Mesh(ctx, lay, params)
    mesh.prim_to_cons(torch.from_numpy(np.ascontiguousarray(W)).to(dev))
    del W
    # let the blast develop before measuring
    for _ in range(20):
        mesh.step(cfl=CFL)
    U0 = mesh.U.clone()
    t0 = mesh.get_time()
    fac, dt0, fmax = mesh.lat_assign(5, CFL, merge_frac=0.0)
    cells = np.array([b[3] * b[4] * b[5] for b in lay.blocks], dtype=np.float64)
    work = float((cells * (fmax // fac)).sum() / (cells.sum() * fmax))
    by_level = {}
    for L in range(3):
        sel = lay.levels == L
        by_level[str(L)] = {str(int(k)): int(((fac == k) & sel).sum()) for k in np.unique(fac[sel])}

    def timed(fn, reps):
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    # LAT window (graph)
    mesh.lat_set_factors(fac, dt0)
    mesh.lat_window(use_graph=True)
    mesh.U.copy_(U0)
    mesh.set_time(t0)
    mesh.lat_set_factors(fac, dt0)
    ms_lat = timed(lambda: mesh.lat_window(use_graph=True), 1)
    rho_lat = mesh.U[0].clone()
    # synchronised steps of dt0 over the same time
    mesh.U.copy_(U0)
    mesh.set_time(t0)
    mesh.step(dt=dt0)   # warm-up (one-factor assignment)
    mesh.U.copy_(U0)
    mesh.set_time(t0)

    def sync_window():
        for _ in range(fmax):
            mesh.step(dt=dt0)
    ms_sync = timed(sync_window, 1)
    flat = torch.from_numpy(lay.interior_flat()).to(dev)
    rl, rs = rho_lat[flat], mesh.U[0][flat]
    drel = (rl - rs).abs() / rs
    ncell = float(cells.sum())
    out = {"workload": "blast wave, 128^3 level-0 grid in 16^3 blocks refined to level 2 within r = 0.15: "
                       "%d blocks (levels 0/1/2: %s), %.2f M cells, PLM + HLLE, dual energy, N_LAT = 5"
                       % (lay.nb, "/".join(str(int(v)) for v in np.bincount(lay.levels)), ncell / 1e6),
           "f_max": int(fmax), "factors_by_level": by_level, "work_fraction": work,
           "ms_lat_window": ms_lat, "ms_sync_same_time": ms_sync, "speedup": ms_sync / ms_lat,
           "ideal_speedup": 1.0 / work,
           "effective_cell_updates_per_s": ncell * fmax / (ms_lat * 1e-3),
           "sync_cell_updates_per_s": ncell * fmax / (ms_sync * 1e-3),
           "rho_lat_vs_sync": {"max_rel": float(drel.max()), "mean_rel": float(drel.mean())},
           "lat_vs_sync_one_window": lat_vs_sync_metrics(torch, rl, rs, params.rho_floor),
           "finite": bool(torch.isfinite(mesh.U).all().item())}
    del mesh, U0
    torch.cuda.empty_cache()
    return out


def remap_bench(ctx, tde, torch, dev, args, n=256, reps=5):
    """Domain remap (Sec. 5.2) of an n^3 dual-energy state in 32^3 MeshBlocks:
    (a) onto an n^3 grid over a domain twice as wide (the debris outgrowing its
    box: an eighth of the target samples the whole source 2x coarser, the rest
    is floor), (b) onto a grid twice as fine, on the half of the source's
    domain with |z| < 1/2 (2n x 2n x n target cells).  Device
    time per remap from CUDA events on the context's stream; algorithmic HBM
    bytes = the source's interior state read once + the target's written."""
    from paper_2609_37859_gb300 import workloads as wl
    src_lay = wl.uniform_layout((n, n, n), (32, 32, 32), ((-1, 1),) * 3, bc=(0, 0, 0), ng=2)
    W = wl.random_smooth(src_lay, seed=SEED, drho=0.5, P0=1.0, modes=4)
    src = tde.Mesh(ctx, src_lay, tde.make_params(dual=1))
    src.prim_to_cons(torch.from_numpy(np.ascontiguousarray(W)).to(dev))
    del W
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    out = {}
    cases = (("enlarge2_coarsen2", (n, n, n), ((-2, 2),) * 3, src_lay.ncells),
             ("refine2_slab", (2 * n, 2 * n, n), ((-1, 1), (-1, 1), (-0.5, 0.5)), src_lay.ncells // 2))
    for name, N, dom, src_cells_read in cases:
        lay = wl.uniform_layout(N, (32, 32, 32), dom, bc=(0, 0, 0), ng=2)
        dst = tde.Mesh(ctx, lay, tde.make_params(dual=1, rho_floor=1e-8, u_floor=1e-10))
        dst.remap_from(src, src.U)   # warm-up
        torch.cuda.synchronize(dev)
        ctx.profile(True)
        for _ in range(reps):
            dst.remap_from(src, src.U)
        prof = ctx.profile_read()
        ctx.profile(False)
        ms_stage = prof["scalar"][1] / reps   # staging and weight tables
        ms_map = prof["remap"][1] / reps
        ms = ms_stage + ms_map
        nbytes = 6 * 8.0 * (src_cells_read + lay.ncells)
        out[name] = {"target_cells": lay.ncells, "ms": ms, "ms_stage": ms_stage, "ms_remap_kernel": ms_map,
                     "target_cells_per_s": lay.ncells / (ms * 1e-3),
                     "algorithmic_bytes": nbytes, "achieved_gbs": nbytes / (ms * 1e-3) * 1e-9,
                     "peak_gbs": hbm, "frac": nbytes / (ms * 1e-3) * 1e-9 / hbm,
                     "finite": bool(torch.isfinite(dst.U).all().item())}
        del dst
        torch.cuda.empty_cache()
    del src
    torch.cuda.empty_cache()
    return {"workload": "%d^3 dual-energy source, 32^3 MeshBlocks, random smooth; thermal-energy form, "
                        "N_qd = 8" % n, "cases": out}


# ------------------------------------------------------ production shape (C5) ---

# rho_floor (rho0), p_floor (rho0 v0^2): 100x Table 1's.  With Table 1's floors
# this unrelaxed star (no self-gravity) leaves non-finite cells in LAT windows:
# floor cells at the star's tip are heated within one step of a slow block (c_s
# 0.13 -> 26) and its fixed step then runs at Courant number 2; with these, none.
C5_FLOORS = (1e-8, 1e-10)
C5_WORKLOAD = ("production-shaped: stretched n=1.5 polytrope (1 Msun, 1 Rsun, 4:1) in its own frame, a 1e3 Msun "
               "point mass with excision passing at the parabolic speed through free-falling ambient gas; "
               "2048 MeshBlocks of 32^3 (512x512x256 = 67,108,864 cells), ghost width 3, PPM+HLLC+SSP-RK2, "
               "Saha H/He 256x256 table in the code units of Table 1, learned-guess closure (BF16 tensor-core "
               "MLP + FP64 Newton, bisection fallback), dual energy, floors 100x Table 1's, CFL 0.3")


def build_c5(ctx, eos, tde, torch, dev, floors=C5_FLOORS, grid=(16, 16, 8)):
    """The production-shaped mesh; `grid` (blocks per axis) other than 16 x 16 x 8
    keeps the cell size and takes the blocks around the star (a smaller case
    of the same workload, for profiling)."""
    from paper_2609_37859_gb300 import workloads as wl
    t0 = time.time()
    half = tuple(n * 32 * 0.0625 / 2.0 for n in grid)   # Rsun: 32-cell blocks of 0.0625 Rsun
    lay, f, bhp = wl.star_c5(seed=SEED, rho_floor=floors[0], p_floor=floors[1], n_blocks=tuple(grid),
                             half_rsun=half)
    W = wl.prim_state(lay, f["rho"], f["vx"], f["vy"], f["vz"], f["P"])
    del f
    params = tde.make_params(eos=tde.EOS_TABLE, recon=tde.RECON_PPM, dual=1, eta1=1e-3, eta2=1e-4,
                             rho_floor=floors[0], p_floor=floors[1], u_floor=1.5 * floors[1],
                             unit_rho=wl.RHO0_CGS, unit_e=wl.V0_CGS ** 2, eos_mode=tde.INVERT_SURROGATE)
    mesh = tde.Mesh(ctx, lay, params, eos)
    mesh.prim_to_cons(torch.from_numpy(W).to(dev))
    del W
    bh = tde.make_bh(on=1, excise=1, GM=bhp["GM"], r_soft=bhp["r_soft"], r_exc=bhp["r_exc"],
                     x0=bhp["x0"], v0=bhp["v0"])
    return lay, mesh, bh, time.time() - t0


def c5_headline(ctx, eos, tde, torch, dev, args, dist, world, barrier, stream):
    """Synchronised steps of the production-shaped mesh (the headline), then the
    same mesh under LAT: windows of f_max fine steps on N_LAT = 6 levels,
    factors re-assigned at every window, replayed as a CUDA graph."""
    lay, mesh, bh, setup_s = build_c5(ctx, eos, tde, torch, dev, grid=args.c5_grid)
    tiles, tile_ms = mesh.autotune(bh=bh, reps=1)
    U_init = mesh.U.clone()
    step = lambda: mesh.step(cfl=CFL, bh=bh)   # noqa: E731
    for _ in range(args.warmup):
        step()
    barrier()
    # the end-to-end steps below start from the state the timed steps start from
    U_t0 = mesh.U.clone()
    mesh.counts(reset=True)
    ctx.profile(True)
    rank, local, _ = dist_env()
    clocks = Clocks(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                    if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.nvtx.range_push("timed_steps")   # lets a profiler select these launches
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile_read()
    clk = clocks.stop()
    ctx.profile(False)
    ms = max_over_ranks(ms, dist, dev)
    counts = mesh.counts(reset=True)
    state_gb = (mesh.U.numel() * 2 + mesh.ntot * (8 + 7)) * 8 / 1e9

    # end to end through the C ABI: the state in from pinned host memory and
    # the result out, every step (each step starts from the initial state)
    host_in = U_t0.cpu().pin_memory()
    del U_t0
    mesh.set_time(0.0)
    run, close, nbytes = e2e_rotating(mesh, host_in, step, torch, dev, stream)
    run(max(1, args.warmup))
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    run(args.steps)
    f1.record(stream)
    barrier()
    ms_e2e = max_over_ranks(f0.elapsed_time(f1), dist, dev)
    close()
    del host_in
    torch.cuda.empty_cache()

    lat = c5_lat(ctx, mesh, lay, bh, U_init, torch, dev) if not args.no_c5 else None
    if lat is not None:
        lat["host_setup_s"] = setup_s
    out = {"ms": ms, "ms_e2e": ms_e2e, "prof": prof, "clocks": clk, "counts": counts, "cells": lay.ncells,
           "meshblocks": lay.nb, "copy_bytes": nbytes, "state_gb": state_gb,
           "autotune": autotune_report(tiles, tile_ms), "lat": lat}
    del mesh, U_init
    torch.cuda.empty_cache()
    return out


def c5_lat(ctx, mesh, lay, bh, U0, torch, dev):
    """LAT on the production-shaped mesh: windows covering 200 fine steps (at
    most 4), factors from the CFL condition at each window start, the captured
    window kept while the level sizes hold; against synchronised steps of dt0."""
    mesh.U.copy_(U0)
    mesh.set_time(0.0)
    fac, dt0, fmax = mesh.lat_assign(6, CFL, merge_frac=0.01, bh=bh)
    cells = np.array([b[3] * b[4] * b[5] for b in lay.blocks], dtype=np.float64)
    work = float((cells * (fmax // fac)).sum() / (cells.sum() * fmax))
    levels = {int(k): int((fac == k).sum()) for k in np.unique(fac)}
    nwin = int(max(1, min(4, -(-200 // fmax))))

    def timed(fn, reps):
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    mesh.lat_set_factors(fac, dt0)
    mesh.lat_window(bh=bh, use_graph=False)   # warm-up: eager, then capture
    mesh.lat_window(bh=bh, use_graph=True)
    # where the first window's time goes: an eager window with CUDA events around
    # every launch, by kernel class, and a synchronised step the same way
    by_kind = {}
    for name, fn in (("lat_window", lambda: mesh.lat_window(bh=bh, use_graph=False)),
                     ("sync_step", lambda: mesh.step(dt=dt0, bh=bh))):
        mesh.U.copy_(U0)
        mesh.set_time(0.0)
        mesh.lat_set_factors(fac, dt0)
        torch.cuda.synchronize(dev)
        ctx.profile(True)
        fn()
        torch.cuda.synchronize(dev)
        by_kind[name] = {k: round(v[1], 3) for k, v in ctx.profile_read().items() if v[0]}
        ctx.profile(False)
    mesh.U.copy_(U0)
    mesh.set_time(0.0)
    mesh.lat_set_factors(fac, dt0)
    mesh.counts(reset=True)
    fmaxes, structures, works = [], set(), []

    def window():
        # as in production: factors from the CFL condition at each window start
        fw, _, fm = mesh.lat_assign(6, CFL, merge_frac=0.01, bh=bh)
        fmaxes.append(int(fm))
        structures.add(tuple(int((fw == k).sum()) for k in (1, 2, 4, 8, 16, 32, 64)))
        works.append(float((cells * (fm // fw)).sum() / (cells.sum() * fm)))
        mesh.lat_window(bh=bh, use_graph=True)
    ms_win = timed(window, nwin)
    c = mesh.counts(reset=True)
    mesh.U.copy_(U0)
    mesh.set_time(0.0)
    mesh.step(dt=dt0, bh=bh)
    ms_step = timed(lambda: mesh.step(dt=dt0, bh=bh), 2)
    ncell = lay.ncells
    return {"workload": "the headline mesh under LAT, N_LAT 6, windows covering 200 fine steps (at most 4)",
            "f_max": int(fmax), "blocks_per_factor": levels,
            "work_fraction": work, "windows": nwin, "fine_steps": nwin * int(fmax),
            "window_f_max": fmaxes, "distinct_level_structures": len(structures),
            "work_fraction_per_window": works,
            "ideal_speedup_timed_windows": 1.0 / float(np.mean(works)),
            "lat_window_ms": ms_win, "sync_step_ms": ms_step, "sync_window_ms_est": ms_step * fmax,
            "lat_speedup_vs_sync": ms_step * np.mean(fmaxes) / ms_win,
            "effective_cell_updates_per_s": ncell * np.mean(fmaxes) / (ms_win * 1e-3),
            "sync_cell_updates_per_s": ncell / (ms_step * 1e-3),
            "floors": {"rho_floor": C5_FLOORS[0], "p_floor": C5_FLOORS[1], "unit": "rho0, rho0 v0^2"},
            "counters_per_window": {k: v // nwin for k, v in c.items()},
            "first_window_ms_by_kernel_class": by_kind}


# ------------------------------------------------------------------ oracle ---

# The oracle's bounded sample of the headline workload: the 4 x 4 x 2 MeshBlocks
# of 32^3 around the star (the same cells, scheme, floors and point mass; the
# point mass lies outside the sample, its potential acts on it).
C5_SAMPLE = dict(n_blocks=(4, 4, 2), half_rsun=(4.0, 4.0, 2.0))


def oracle_c5_sample():
    from oracle import tref
    from paper_2609_37859_gb300 import workloads as wl
    d = np.load(TABLE)
    ot = tref.EOSTable(int(d["n_rho"]), int(d["n_T"]), tuple(d["lrho"]), tuple(d["lT"]),
                       d["log10_e"], d["log10_P"], d["log10_cs2"])
    lay, f, bhp = wl.star_c5(seed=SEED, rho_floor=C5_FLOORS[0], p_floor=C5_FLOORS[1], **C5_SAMPLE)
    W = wl.prim_state(lay, f["rho"], f["vx"], f["vy"], f["vz"], f["P"])
    p = tref.make_params(eos=tref.EOS_TABLE, recon=tref.PPM, dual=1, eta1=1e-3, eta2=1e-4,
                         rho_floor=C5_FLOORS[0], p_floor=C5_FLOORS[1], u_floor=1.5 * C5_FLOORS[1],
                         unit_rho=wl.RHO0_CGS, unit_e=wl.V0_CGS ** 2, bh_on=1, excision_on=1,
                         GM=bhp["GM"], r_soft=bhp["r_soft"], r_exc=bhp["r_exc"], bh_x0=bhp["x0"],
                         bh_v0=bhp["v0"], bh_a0=(0.0, 0.0, 0.0))
    m = tref.Mesh(lay, p, ot)
    U = m.prim_to_cons(W)
    return tref, m, U, lay


class OracleStepper:
    """One step of the oracle on the sample: CFL dt over every block (as the
    GPU step computes it), then the synchronised RK2 step (ghost fill, two
    stages, excision, resync) of every block of the sample."""

    def __init__(self):
        self.tref, self.m, self.U, self.lay = oracle_c5_sample()
        self.S = self.m.new_state()
        self.t = 0.0
        self.cells = self.lay.ncells

    def __call__(self):
        nb = self.lay.nb
        dt = float(self.m.cfl_dt(self.U, CFL, np.full(nb, self.t)).min())
        self.m.step(self.U, dt, self.t, self.S)
        self.t += dt


SAMPLE_NOTE = ("the 4x4x2 MeshBlocks of 32^3 (1,048,576 cells) around the star of the same workload, same "
               "cells, scheme and floors; each step: CFL dt over the sample, then one synchronised RK2 step of "
               "all its MeshBlocks (OpenMP over MeshBlocks, 32 blocks on the host's threads)")


def cpu_baseline(seconds):
    """The oracle as it stands, on the host cores, on a bounded sample of the
    headline workload, for about `seconds`, then on one thread for a third of that."""
    st = OracleStepper()
    tref = st.tref
    st()   # first touch
    n, t0 = 0, time.perf_counter()
    while True:
        st()
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    cores = tref.num_threads()
    tref.set_num_threads(1)
    n1, t1 = 0, time.perf_counter()
    while True:
        st()
        n1 += 1
        el1 = time.perf_counter() - t1
        if el1 >= seconds / 3.0:
            break
    tref.set_num_threads(cores)
    v, v1 = n * st.cells / el, n1 * st.cells / el1
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d steps of %s, %.1f s" % (n, SAMPLE_NOTE, el),
            "threads_busy": min(cores, st.lay.nb),
            "single_thread": {"value": v1, "unit": UNIT, "steps": n1, "seconds": el1},
            "all_thread_speedup": v / v1}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    st = OracleStepper()
    for _ in range(args.warmup):
        st()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st()
    el = time.perf_counter() - t0
    v = args.steps * st.cells / el
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": C5_WORKLOAD, "cells_per_step": st.cells},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": st.tref.num_threads(), "kind": "oracle",
                         "sample": "each step: " + SAMPLE_NOTE},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--no-c5", action="store_true", help="skip LAT windows on the headline mesh")
    ap.add_argument("--no-grav", action="store_true", help="skip the self-gravity multigrid")
    ap.add_argument("--no-remap", action="store_true", help="skip the domain remap")
    ap.add_argument("--remap-n", type=int, default=256, help="source grid of the remap section (n^3)")
    ap.add_argument("--no-smr", action="store_true", help="skip LAT on the refined blast-wave mesh")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-eos", action="store_true", help="skip the EOS-inversion comparison")
    ap.add_argument("--no-lat", action="store_true", help="skip the LAT stream comparison")
    ap.add_argument("--no-c2", action="store_true", help="skip the entropy-wave (128^3) section")
    ap.add_argument("--no-headline", action="store_true",
                    help="profiling: run only the EOS-inversion and self-gravity sections (no headline line)")
    ap.add_argument("--c5-grid", type=lambda v: tuple(int(x) for x in v.split(",")), default=(16, 16, 8),
                    help="MeshBlocks per axis of the headline mesh (profiling cases; default 16,16,8)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
