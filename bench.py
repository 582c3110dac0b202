#!/usr/bin/env python
"""Benchmark: abstract-rendering throughput in pixel x pose-cell bounds per second.

One step = one abstract render of the whole workload (every pose cell, every
pixel: pose prep, record prep with MatrixInv, binning, per-pixel relaxation and
BlendInd) through the C ABI.  The default workload is the 300k-Gaussian object
scene at 800x800 with a 6-DoF box split into 64 cells.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank renders its own copy
of the workload (weak scaling, no collective on the data path); the time is
the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pixel x pose-cell bounds/s"
UNIT = "pixel-cells/s"
SMS, FP32_LANES, MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * MAX_MHZ * 1e6 / 1e12   # FMA = 2 flops

# FP32 operations of the relaxation itself per evaluated (pixel, Gaussian,
# cell) triple, with M pose variables (an FMA = 2 flops, any other FP32
# operation = 1, expf = 2: a multiply and the SFU exponential):
#   Delta_x, Delta_y = (u - mu) S + R          4 M + 8
#   concretising Delta_x, Delta_y, q0..q2, m   6 M + 12   (k -+ sum |c|)
#   q_c: 6 averaged-McCormick products        24 M + 132
#   m = sum q_c^2: 3 tangent/secant squares    6 M + 45
#   Exp (Table 2), opacity, clip and cutoff    6 M + 60
#   both colour sums (lower and upper endpoint) and the transmittances
#                                             12 M + 26
# = 58 M + 283 (631 at M = 6).  The rounding-error bookkeeping that keeps the
# FP32 bounds sound (the gamma_n sum |a| r terms, midpoint slacks, widened
# exps, the colour sums' error bounds) is about 156 more and is not counted.
def flops_per_triple(M: int) -> int:
    return 58 * M + 283


BOOKKEEPING_FLOPS_PER_TRIPLE = 156


# DRAM bytes of the render kernel per opacity evaluation, from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of round 0 of the first 4
# cells of the 300k-Gaussian workload, both instances (FP32 sweep 35.6 MB, FP64
# re-sweep 15.0 MB), over the render's 73.2M evaluations.  Valid only for the
# kernel sources it was taken from (their SHA-256 below); otherwise the
# roofline's traffic is reported as null.
RENDER_TRAFFIC = {"bytes_per_evaluation": (27421952 + 8210688 + 14208256 + 770304) / 73160149,
                  # the same capture's smsp__issue_active of the FP32 sweep (the bound of
                  # this issue-limited kernel: one warp instruction per scheduler per cycle)
                  "issue_active_fp32_sweep": 0.6353,
                  "sources": ["k_render.cuh", "ar_num.cuh", "ar_common.cuh", "k_inst.cuh"],
                  "sha256": "8c9745917e963b6bda2abd316fbede1feb72bca27086a702d94f1fa9fdf3beea"}


def render_capture_valid() -> bool:
    import hashlib
    h = hashlib.sha256()
    for f in RENDER_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, "paper_2503_00308_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest() == RENDER_TRAFFIC["sha256"]


def render_traffic(n_evaluated: int):
    if not render_capture_valid():
        return None
    return RENDER_TRAFFIC["bytes_per_evaluation"] * n_evaluated


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="object300k")
    ap.add_argument("--tile", type=int, default=0, help="0: the library's autotuner picks the tile edge")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-window", type=int, default=32,
                    help="edge of the oracle's pixel sample (32: about 15 s of oracle work on 16 cores)")
    ap.add_argument("--cells", type=int, default=0, help="use only the first N cells (profiling slices)")
    ap.add_argument("--relational-steps", type=int, default=2,
                    help="timed steps of the relational-transmittance blend (0: skip)")
    ap.add_argument("--serve-requests", type=int, default=32, help="requests in the serving mix (0: skip)")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=96.0)
    ap.add_argument("--serve-load", type=float, default=0.9,
                    help="offered load of the Poisson stream, as a fraction of the one-at-a-time capacity")
    ap.add_argument("--plain-cells", type=int, default=1,
                    help="cells timed through the plain FP64 one-cell-per-launch path (0: skip)")
    ap.add_argument("--workloads", default="object10k,unbounded750k",
                    help="further workloads timed beside the main one ('' to skip)")
    ap.add_argument("--workload-steps", type=int, default=2)
    ap.add_argument("--sound-poses", type=int, default=16,
                    help="concrete renders of cell 0 checked against the timed bounds (0: skip)")
    ap.add_argument("--no-small-cells", action="store_true")
    return ap.parse_args()


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return rank, world, local, pg


def max_over_ranks(x: float, pg) -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    if pg is None:
        return x
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Units all ranks processed per second, timed by the slowest rank."""
    return units_per_rank * world / (ms_max / 1e3)


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def centre_window(w, window_edge: int):
    cx, cy = w.camera.width // 2, w.camera.height // 2
    h = window_edge // 2
    return (cx - h, cx - h + window_edge - 1, cy - h, cy - h + window_edge - 1)


def cpu_baseline(w, window_edge: int, cell: int = 0, keep=None):
    """Time the FP64 oracle (as it stands) on a pixel window of one cell.  With
    keep (a dict), the oracle's bounds of the window are left in it, for the
    accuracy of the GPU's bounds there."""
    import oracle
    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    win = centre_window(w, window_edge)
    t0 = time.perf_counter()
    r = oracle.render_abstract(w.scene, w.camera, w.cells_lo[cell], w.cells_hi[cell], window=win)
    dt = time.perf_counter() - t0
    if keep is not None:
        keep.update(cell=cell, window=win, lo=r[0], hi=r[1], frag=r[2])
    units = window_edge * window_edge
    return {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%dx%d pixels at the image centre (densest region) of cell %d of %s; %.1f s" %
                      (window_edge, window_edge, cell, w.name, dt)}


def accuracy(orc_out, glo, ghi):
    """GPU bounds of one cell against the oracle's on its window: the largest
    |gpu - oracle| over channels at non-fragile pixels, how many pixels exceed
    the 1e-4 contract, the fragile fraction."""
    import numpy as np
    olo, ohi, frag = orc_out["lo"], orc_out["hi"], orc_out["frag"]
    m = ~np.isnan(olo[..., 0])
    ok = m & (frag == 0)
    e = np.maximum(np.abs(glo - olo), np.abs(ghi - ohi)).max(axis=-1)
    x0, x1, y0, y1 = orc_out["window"]
    return {"cell": int(orc_out["cell"]), "window": "%dx%d at (%d, %d)" % (x1 - x0 + 1, y1 - y0 + 1, x0, y0),
            "pixels": int(ok.sum()), "max_abs_err": float(e[ok].max(initial=0.0)),
            "n_over_1e-4": int((e[ok] > 1e-4).sum()),
            "fragile_frac": float((m & (frag != 0)).sum()) / max(1, int(m.sum()))}


def gap_metrics(lo, hi):
    """MPG and XPG of the paper's evaluation: the mean and the largest over
    pixels of the RGB norm of upper - lower (per cell, then averaged over the
    cells for MPG and maximised for XPG); device tensors [n][H][W][3]."""
    g = (hi.double() - lo.double()).norm(dim=-1)
    return {"mpg": float(g.mean()), "xpg": float(g.max())}


def soundness(ar, s, w, out_lo, out_hi, n_poses, sp, cell=0):
    """Concrete FP64 renders on the device (ar_render_concrete) at the cell's
    two extreme corners and n_poses - 2 seeded random poses of the cell: the
    number of (pose, pixel, channel) values outside the GPU bounds of the
    timed step, with no tolerance."""
    import numpy as np
    import torch

    from paper_2503_00308_gb300 import synth
    lo, hi = w.cells_lo[cell], w.cells_hi[cell]
    poses = np.concatenate([lo[None], hi[None],
                            synth.sample_poses(np.random.default_rng(7), lo, hi, max(0, n_poses - 2))])
    cam = w.camera
    img = torch.empty((1, cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    bad = 0
    for p in poses:
        s.render_concrete(cam, p[None], img, sp)
        torch.cuda.synchronize()
        bad += int(((img[0] < out_lo[cell]) | (img[0] > out_hi[cell])).sum())
    return {"cell": cell, "poses": int(len(poses)), "violations": bad, "values_checked": int(len(poses)) * img.numel()}


def run_reference(args, rank):
    if rank != 0:
        return
    from paper_2503_00308_gb300 import synth
    w = synth.WORKLOADS[args.workload]()
    for _ in range(args.warmup):
        cpu_baseline(w, max(4, args.cpu_window // 2))
    vals = []
    t0 = time.perf_counter()
    for s in range(args.steps):
        vals.append(cpu_baseline(w, args.cpu_window, cell=s % w.n_cells))
    total = time.perf_counter() - t0
    v = statistics.median([x["value"] for x in vals])
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "gaussians": w.scene.n, "image": "%dx%d" % (w.camera.width, w.camera.height),
                       "cells": w.n_cells, "sample": vals[0]["sample"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def plain_path(ar, s, w, intr, pose, args, sp, value):
    """The plain FP64 path (one cell per launch sequence, FP64 records and
    per-pixel arithmetic, no early stopping) on the first cells of the same
    workload; one untimed run, then one timed with CUDA events."""
    import torch
    k = min(args.plain_cells, w.n_cells)
    cam = w.camera
    cells = ar.make_cells(w.cells_lo[:k], w.cells_hi[:k])
    o_lo = torch.empty((k, cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    o_hi = torch.empty_like(o_lo)
    stream = torch.cuda.current_stream()
    ar.ar_render_abstract_plain_fp64(s.handle, intr, pose, cells, k, args.tile, o_lo, o_hi, sp)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ar.ar_render_abstract_plain_fp64(s.handle, intr, pose, cells, k, args.tile, o_lo, o_hi, sp)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    st = ar.ar_last_render_stats(s.handle)
    pv = k * cam.width * cam.height / (ms / 1e3)
    return {"value": pv, "unit": UNIT, "cells": k, "ms": ms, "dtype": "f64", "warmup": 1, "steps": 1,
            "stages_ms": {"prep": st["ms_prep"], "bin": st["ms_bin"], "render": st["ms_render"]},
            "speedup": value / pv}


def relational(ar, s, w, intr, pose, cells, nc, args, sp, out_lo, out_hi, value):
    """The relational upper transmittance (AR_BLEND_RELATIONAL) on the same
    workload: W warm-up and K timed steps with CUDA events, the mean bounds of
    both blends (out_lo / out_hi hold the interval blend's last step), and the
    same on the first cell shrunk to a twentieth of its widths, where the bounds
    are no longer saturated."""
    import numpy as np
    import torch
    stream = torch.cuda.current_stream()
    mean_int = (float(out_lo.double().mean()), float(out_hi.double().mean()))
    ar.ar_scene_set_blend(s.handle, ar.AR_BLEND_RELATIONAL)
    try:
        for _ in range(args.warmup):
            ar.ar_render_abstract(s.handle, intr, pose, cells, nc, args.tile, out_lo, out_hi, sp)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.relational_steps):
            ar.ar_render_abstract(s.handle, intr, pose, cells, nc, args.tile, out_lo, out_hi, sp)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.relational_steps
        st = ar.ar_last_render_stats(s.handle)
        mean_rel = (float(out_lo.double().mean()), float(out_hi.double().mean()))
        # one small cell: the first cell's centre with a twentieth of its widths
        c = 0.5 * (w.cells_lo[0] + w.cells_hi[0])
        h = 0.025 * (w.cells_hi[0] - w.cells_lo[0])
        small = ar.make_cells((c - h)[None], (c + h)[None])
        cam = w.camera
        o_lo = torch.empty((1, cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
        o_hi = torch.empty_like(o_lo)
        widths = {}
        for name, mode in (("interval", ar.AR_BLEND_INTERVAL), ("relational", ar.AR_BLEND_RELATIONAL)):
            ar.ar_scene_set_blend(s.handle, mode)
            ar.ar_render_abstract(s.handle, intr, pose, small, 1, args.tile, o_lo, o_hi, sp)
            torch.cuda.synchronize()
            widths[name] = float((o_hi - o_lo).double().mean())
    finally:
        ar.ar_scene_set_blend(s.handle, ar.AR_BLEND_INTERVAL)
    pv = w.pixel_cells() / (ms / 1e3)
    return {"value": pv, "unit": UNIT, "ms_per_step": ms, "warmup": args.warmup, "steps": args.relational_steps,
            "vs_interval": pv / value, "render_ms": st["ms_render"], "evaluated": st["n_evaluated"],
            "mean_lower": {"interval": mean_int[0], "relational": mean_rel[0]},
            "mean_upper": {"interval": mean_int[1], "relational": mean_rel[1]},
            "small_cell_mean_width": widths}


def timed_render(ar, s, intr, pose, cells, nc, tile, out_lo, out_hi, sp, warmup, steps):
    """W untimed and K timed renders (CUDA events on the stream); ms per step and the last stats."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        ar.ar_render_abstract(s.handle, intr, pose, cells, nc, tile, out_lo, out_hi, sp)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    render_ms = []
    for _ in range(steps):
        ar.ar_render_abstract(s.handle, intr, pose, cells, nc, tile, out_lo, out_hi, sp)
        render_ms.append(ar.ar_last_render_stats(s.handle)["ms_render"])
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / steps, ar.ar_last_render_stats(s.handle), statistics.mean(render_ms)


def roofline_of(stats, r_ms):
    M = stats["m_vars"]
    flops = flops_per_triple(M) * stats["n_evaluated"]
    achieved = flops / (r_ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS, "kernel": "render_kernel", "kernel_ms": r_ms,
            "flops_per_triple": flops_per_triple(M), "triples_evaluated": stats["n_evaluated"]}


def stage_dict(st):
    return {"prep": st["ms_prep"], "bin": st["ms_bin"], "build": st["ms_build"], "render": st["ms_render"],
            "total": st["ms_total"]}


def count_dict(st):
    return {"records": st["n_records"], "entries": st["n_entries"], "triples": st["n_triples"],
            "evaluated": st["n_evaluated"], "reevaluated": st["n_reevaluated"], "fallback": st["n_fallback"],
            "split": st["n_split"], "built": st["n_built"], "restarted": st["n_restarted"],
            "fp64_evaluations": st["n_fp64"], "fp64_segments": st["n_fp64_segments"]}


def workload_leg(ar, name, args, sp, warmup, steps, window_edge):
    """Another workload of the paper's shapes through the same call: throughput,
    stages, counts, the render kernel's roofline, MPG/XPG and the accuracy
    against the oracle on a window of cell 0 at the image centre."""
    import torch

    from paper_2503_00308_gb300 import synth
    w = synth.WORKLOADS[name]()
    cam, nc = w.camera, w.n_cells
    s = ar.Scene(w.scene)
    ar.ar_set_profiling(s.handle, True)
    intr, pose, cells = ar.make_intrinsics(cam), ar.make_pose(cam), ar.make_cells(w.cells_lo, w.cells_hi)
    out_lo = torch.empty((nc, cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    out_hi = torch.empty_like(out_lo)
    ms, st, r_ms = timed_render(ar, s, intr, pose, cells, nc, args.tile, out_lo, out_hi, sp, warmup, steps)
    keep = {}
    cpu = cpu_baseline(w, window_edge, keep=keep)
    glo = out_lo[0].double().cpu().numpy()
    ghi = out_hi[0].double().cpu().numpy()
    acc = accuracy(keep, glo, ghi)
    out = {"value": w.pixel_cells() / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "warmup": warmup, "steps": steps,
           "config": {"workload": w.name, "gaussians": w.scene.n, "image": "%dx%d" % (cam.width, cam.height),
                      "cells": nc, "pose_vars": st["m_vars"], "tile": st["tile"], "chunk": st["chunk"]},
           "stages_ms": stage_dict(st), "counts": count_dict(st), "roofline": roofline_of(st, r_ms),
           "gaps": gap_metrics(out_lo, out_hi), "accuracy": acc, "oracle_sample": cpu["sample"]}
    s.close()
    return out


def small_cells_leg(ar, s, w, intr, pose, args, sp, out_lo, out_hi):
    """The benchmark workload with every cell shrunk about its centre to a
    twentieth of its widths, so that the bounds are informative instead of
    saturated: throughput, evaluations per in-box triple, the render kernel's
    roofline and MPG/XPG."""
    import numpy as np
    c = 0.5 * (w.cells_lo + w.cells_hi)
    h = 0.025 * (w.cells_hi - w.cells_lo)
    nc = w.n_cells
    cells = ar.make_cells(c - h, c + h)
    ms, st, r_ms = timed_render(ar, s, intr, pose, cells, nc, args.tile, out_lo, out_hi, sp, args.warmup,
                                max(1, min(args.steps, 3)))
    return {"value": w.pixel_cells() / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "cells": "the %d benchmark cells, each shrunk about its centre to 1/20 of its widths" % nc,
            "stages_ms": stage_dict(st), "counts": count_dict(st),
            "evaluations_per_triple": st["n_evaluated"] / max(1, st["n_triples"]),
            "roofline": roofline_of(st, r_ms), "gaps": gap_metrics(out_lo, out_hi),
            "mean_width": float((out_hi - out_lo).double().mean())}


def fma_probe(sp):
    """Measured FP32 FMA rate, scalar and packed (best of 3 each), beside the nominal peak
    (the benchmark's own helper library, not libar)."""
    from paper_2503_00308_gb300 import probe
    out = {}
    for name, packed in (("scalar", False), ("packed", True)):
        out[name] = max(probe.fp32_fma_rate(packed, 16384, sp) for _ in range(3))
    return out


def hbm_peak():
    """Measured HBM copy bandwidth (GB/s) of this machine's GPUs, else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def union_leg(ar, w, nc, args, sp, out_lo, out_hi):
    """ar_bounds_union over the workload's cells (the bounds of the whole pose
    box): W warm-ups and K timed launches with CUDA events.  The inputs (both
    bound images of every cell) are far larger than L2."""
    import torch
    cam = w.camera
    stream = torch.cuda.current_stream()
    u_lo = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    u_hi = torch.empty_like(u_lo)
    for _ in range(args.warmup):
        ar.ar_bounds_union(out_lo, out_hi, nc, cam.width, cam.height, u_lo, u_hi, sp)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        ar.ar_bounds_union(out_lo, out_hi, nc, cam.width, cam.height, u_lo, u_hi, sp)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    n = cam.height * cam.width * 3
    nbytes = 4 * (2 * nc * n + 2 * n)
    peak, src = hbm_peak()
    gbs = nbytes / (ms / 1e3) / 1e9
    return {"ms": ms, "bytes_per_launch": nbytes, "achieved_gbs": gbs, "peak_gbs": peak, "peak_source": src,
            "frac": gbs / peak, "launches": args.steps, "mean_width": float((u_hi - u_lo).double().mean())}


def serving(ar, args, sp):
    """The serving mix: a seeded Poisson stream of requests over resident
    10k / 300k / 750k-Gaussian scenes (200x200 to 1280x720, 1 to 256 cells).

    (1) one request at a time, closed loop, through ar_render_abstract: the
        plain one-request-per-launch path; its mean service time sets the
        arrival rate (offered load = --serve-load of its capacity);
    (2) the same arrival stream through a one-slot server (no overlap);
    (3) the same stream through an --serve-slots server (continuous batching);
    (4) capacity: every request submitted at once, to both servers.
    Latency is submit-to-completion, measured by the server."""
    import numpy as np
    import torch

    from paper_2503_00308_gb300 import synth
    reqs = synth.serving_mix(args.serve_requests, seed=0)
    scenes = {k: ar.Scene(synth.SERVE_SCENES[k]()) for k in sorted({q.scene for q in reqs})}
    outs = []
    for q in reqs:
        o = torch.empty((q.cells_lo.shape[0], q.camera.height, q.camera.width, 3), dtype=torch.float32,
                        device="cuda")
        outs.append((o, torch.empty_like(o)))
    units = [q.pixel_cells() for q in reqs]
    # warm-up: the largest request of each scene
    for k, sc in scenes.items():
        i = max((j for j, q in enumerate(reqs) if q.scene == k), key=lambda j: units[j])
        sc.render(reqs[i].camera, reqs[i].cells_lo, reqs[i].cells_hi, outs[i][0], outs[i][1], stream=sp)
    torch.cuda.synchronize()
    service = []
    for q, (a, b) in zip(reqs, outs):
        t0 = time.perf_counter()
        scenes[q.scene].render(q.camera, q.cells_lo, q.cells_hi, a, b, stream=sp)
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t0)
    total = float(sum(units))
    mean_gap = statistics.mean(service) / args.serve_load
    arrivals = np.cumsum([q.gap * mean_gap for q in reqs])
    arrivals -= arrivals[0]

    def stream(slots, burst=False):
        at = np.zeros_like(arrivals) if burst else arrivals
        srv = ar.Server(int(args.serve_budget_gb * (1 << 30)), slots)
        lat, end = [None] * len(reqs), [None] * len(reqs)
        pending, i = {}, 0
        t0 = time.perf_counter()
        while i < len(reqs) or pending:
            now = time.perf_counter() - t0
            while i < len(reqs) and at[i] <= now:
                q = reqs[i]
                t = srv.submit(scenes[q.scene], q.camera, q.cells_lo, q.cells_hi, outs[i][0], outs[i][1])
                assert t is not None
                pending[t] = i
                i += 1
            for t in list(pending):
                done, ms = srv.poll(t)
                if done:
                    lat[pending[t]] = ms
                    end[pending[t]] = time.perf_counter() - t0
                    del pending[t]
            time.sleep(0.0002)
        srv.close()
        span = max(end)
        out = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
               "mean_ms": float(np.mean(lat)), "bounds_per_s": total / span, "makespan_s": span}
        # latency per request-size class: at most 4 cells (high priority in
        # the server) and more
        for name, sel in (("small", [q.cells_lo.shape[0] <= 4 for q in reqs]),
                          ("large", [q.cells_lo.shape[0] > 4 for q in reqs])):
            ls = [x for x, k in zip(lat, sel) if k]
            if ls:
                out[name] = {"requests": len(ls), "p50_ms": float(np.percentile(ls, 50)),
                             "p99_ms": float(np.percentile(ls, 99))}
        return out

    one = stream(1)
    many = stream(args.serve_slots)
    one_b = stream(1, burst=True)
    many_b = stream(args.serve_slots, burst=True)
    for sc in scenes.values():
        sc.close()
    return {"requests": len(reqs), "pixel_cells": int(total), "slots": args.serve_slots,
            "budget_gb": args.serve_budget_gb, "offered_load": args.serve_load,
            "mean_interarrival_ms": mean_gap * 1e3, "unit": UNIT,
            "one_at_a_time_closed_loop": {"bounds_per_s": total / sum(service),
                                          "p50_service_ms": float(np.percentile(service, 50) * 1e3),
                                          "p99_service_ms": float(np.percentile(service, 99) * 1e3)},
            "one_slot_server": one, "continuous_batching": many,
            "saturated": {"one_slot_bounds_per_s": one_b["bounds_per_s"],
                          "continuous_batching_bounds_per_s": many_b["bounds_per_s"],
                          "one_slot_makespan_s": one_b["makespan_s"],
                          "continuous_batching_makespan_s": many_b["makespan_s"]},
            "p50_ms": many["p50_ms"], "p99_ms": many["p99_ms"], "bounds_per_s": many["bounds_per_s"]}


def run_ours(args, rank, world, local, pg):
    import numpy as np
    import torch

    from paper_2503_00308_gb300 import _build, ar, synth
    if local == 0 or not os.path.exists(_build.LIB):
        _build.build()
    if pg is not None:
        pg.barrier()
    torch.cuda.set_device(local)
    w = synth.WORKLOADS[args.workload]()
    if args.cells:
        w.cells_lo, w.cells_hi = w.cells_lo[:args.cells], w.cells_hi[:args.cells]
        w.name += "[%d cells]" % w.n_cells
    cam = w.camera
    nc = w.n_cells
    s = ar.Scene(w.scene)
    ar.ar_set_profiling(s.handle, True)
    intr, pose = ar.make_intrinsics(cam), ar.make_pose(cam)
    cells = ar.make_cells(w.cells_lo, w.cells_hi)
    out_lo = torch.empty((nc, cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    out_hi = torch.empty_like(out_lo)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def step():
        ar.ar_render_abstract(s.handle, intr, pose, cells, nc, args.tile, out_lo, out_hi, sp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    time.sleep(0.3 if clocks else 0)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    render_ms, stats = [], None
    for _ in range(args.steps):
        step()
        stats = ar.ar_last_render_stats(s.handle)
        render_ms.append(stats["ms_render"])
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, pg)
    if pg is not None:
        pg.barrier()
    units = w.pixel_cells() * world
    value = whole_job_rate(w.pixel_cells(), world, ms)

    # end to end through the host-buffer entry point: per step the pose cells
    # go host -> device and both bound images come back device -> host
    e2e = None
    if not args.no_e2e:
        h_lo = torch.empty(out_lo.shape, dtype=torch.float32, pin_memory=True)
        h_hi = torch.empty_like(h_lo, pin_memory=True)
        for _ in range(args.warmup):
            ar.ar_render_abstract_host(s.handle, intr, pose, cells, nc, args.tile, h_lo, h_hi, sp)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ar.ar_render_abstract_host(s.handle, intr, pose, cells, nc, args.tile, h_lo, h_hi, sp)
        dt = max_over_ranks((time.perf_counter() - t0) / args.steps, pg)
        e2e = {"value": units / dt, "unit": UNIT, "h2d_bytes_per_step": nc * 96,
               "d2h_bytes_per_step": 2 * out_lo.numel() * 4,
               "d2h": "render kernel stores into the mapped page-locked host buffers (overlapped)"}
    if rank != 0:
        return
    M = stats["m_vars"]
    flops = flops_per_triple(M) * stats["n_evaluated"]
    r_ms = statistics.mean(render_ms)
    achieved = flops / (r_ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "gaussians": w.scene.n, "image": "%dx%d" % (cam.width, cam.height),
                   "cells": nc, "pose_vars": M, "tile": stats["tile"], "chunk": stats["chunk"],
                   "tile_choice": ("autotuned over (tile, chunk) in (16, 16), (16, 8), (16, 32), (8, 16)"
                                   if args.tile == 0 else "fixed"),
                   "l2": "working set (records + bins, tens of GB) far larger than L2; no flush needed"},
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": int(stats["n_launches"]) * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": render_traffic(stats["n_evaluated"]),
                     "traffic_unit": "DRAM bytes per render step (all render_kernel launches of the step)",
                     "kernel": "render_kernel", "kernel_ms": r_ms,
                     "flops_per_triple": flops_per_triple(M),
                     "flops_note": "the relaxation's own FP32 arithmetic (FMA = 2, other ops = 1, expf = 2); "
                                   "%d more of rounding-error bookkeeping per triple not counted; kernel_ms "
                                   "is both render instances (FP32 sweep and FP64 re-sweep)"
                                   % BOOKKEEPING_FLOPS_PER_TRIPLE,
                     "triples_evaluated": stats["n_evaluated"],
                     "triples_in_boxes": stats["n_triples"],
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (nominal: MEASURED_PEAKS.json has no FP32 figure)",
                     "fp32_fma_probe_tflops": fma_probe(sp),
                     "issue_active_fp32_sweep": (RENDER_TRAFFIC["issue_active_fp32_sweep"]
                                                 if render_capture_valid() else None),
                     "issue_note": "ncu smsp__issue_active of the FP32 sweep on the first 4 cells, from the "
                                   "capture the traffic figure comes from: the kernel is bound by instruction "
                                   "issue (directed-rounding bookkeeping), not by FP32 FLOPs"},
        "stages_ms": {"prep": stats["ms_prep"], "bin": stats["ms_bin"], "build": stats["ms_build"],
                      "render": stats["ms_render"], "total": stats["ms_total"]},
        "counts": count_dict(stats),
        "gaps": gap_metrics(out_lo, out_hi),
    }
    if args.sound_poses > 0:
        line["soundness"] = soundness(ar, s, w, out_lo, out_hi, args.sound_poses, sp)
    keep = {}
    if not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_window, keep=keep)
        line["accuracy"] = accuracy(keep, out_lo[keep["cell"]].double().cpu().numpy(),
                                    out_hi[keep["cell"]].double().cpu().numpy())
    line["union"] = union_leg(ar, w, nc, args, sp, out_lo, out_hi)
    if args.relational_steps > 0:
        line["relational"] = relational(ar, s, w, intr, pose, cells, nc, args, sp, out_lo, out_hi, value)
    if args.plain_cells > 0:
        line["plain_path"] = plain_path(ar, s, w, intr, pose, args, sp, value)
    if not args.no_small_cells:
        line["small_cells"] = small_cells_leg(ar, s, w, intr, pose, args, sp, out_lo, out_hi)
    s.close()
    if args.serve_requests > 0:
        line["serving"] = serving(ar, args, sp)
    if args.workloads and world == 1:
        line["workloads"] = {}
        for name in [x for x in args.workloads.split(",") if x and x != args.workload]:
            line["workloads"][name] = workload_leg(ar, name, args, sp, max(1, min(args.warmup, 2)),
                                                   args.workload_steps, 32 if name == "object10k" else 16)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
