"""Benchmark of the batched ENUFFT type-1 + EMS hot path on B300 (one JSON line on stdout).

A step is one pass of the whole hot path over the batch: per-cell window/scale, spread, 2-D FFT,
deconvolve/crop and Elastic Mode Selection of every cell (enufft_type1_ems).  Inputs are synthetic
(seeded generator `synth`), resident in HBM for `value`; `e2e` times the same call with host
buffers, the host-to-device copy of the samples and the device-to-host read of the EMS result inside
the timed region.  `--impl reference` times the FP64 CPU oracle (a deliberately plain program) on a
bounded sample of the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "NU points/s, batched type-1 ENUFFT+EMS at rel-l2<=1e-5; mixed vs plain FP32, 1 B300"
# compute peaks of this GPU from `python bench.py --peaks` (enufft_probe_peaks): binary32 FMA TFLOP/s
# and conflict-free shared-memory 32-bit reductions per second (1e9) over all SMs
FP32_TFLOPS = 70.9
SMEM_RED_GOPS = 9120.0
DEFAULT_WORKLOAD = "tri81920_p64_mixed"
KERNEL_SOURCES = ["common.cuh", "fft.cuh", "ems.cuh", "forward.cuh", "inst_common.cuh", "inst_f32_128.cu"]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


def _kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2606_21278_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(workload):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(workload)
    if not e or e.get("kernel_hash") != _kernel_hash():
        return None
    return e.get("dram_bytes_per_launch")


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([s.strip() for s in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.t.join(timeout=2)

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 8 for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank


def _barrier(ws):
    if ws > 1:
        torch.distributed.barrier()


def _reduce_device():
    """Device of the scalar reductions: the GPU under NCCL, the host under gloo."""
    if torch.distributed.is_initialized() and torch.distributed.get_backend() == "nccl":
        return "cuda"
    return "cpu"


def _max_over_ranks(v, ws):
    if ws == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=_reduce_device())
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(v, ws):
    if ws == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=_reduce_device())
    torch.distributed.all_reduce(t)
    return float(t.item())


def _oracle_sample(wl_cpu_fn, target_s=15.0):
    """Time the FP64 oracle (type-1 + EMS) on a growing seeded sample of cells until ~target_s of CPU
    work; returns points/s, cells, points, threads, seconds."""
    import oracle
    wl = wl_cpu_fn()
    rng = np.random.default_rng(0)
    perm = rng.permutation(wl.n_cells)
    n = 4
    while True:
        sub = wl.cell_slice(sorted(perm[:n].tolist()))
        t0 = time.perf_counter()
        c = oracle.type1(sub)
        oracle.ems(c)
        dt = time.perf_counter() - t0
        if dt > target_s / 4 or n >= wl.n_cells:
            break
        n = min(wl.n_cells, int(n * max(2.0, min(8.0, target_s / 4 / max(dt, 1e-3)))))
    return sub.n_points / dt, sub.n_cells, sub.n_points, oracle.threads_used(), dt


def _workload(args, seed, device):
    """The named synthetic workload, optionally resized (--cells, --q-scale), with cells capped at
    --max-q samples and the tensor-core routing threshold overridden by --tc-max-points."""
    wl = synth.make(args.workload, seed=seed, device=device, n_cells=args.cells, q_scale=args.q_scale)
    if args.max_q is not None:
        wl = wl.truncated(args.max_q)
    if args.tc_max_points is not None:
        wl.tc_max_points = args.tc_max_points
    wl.frame = 1 if getattr(args, "frame", "centroid") == "edge" else 0
    return wl


def _rank_workload(args, ws, rank, device):
    """This rank's share of the job.  The job is one seeded batch made of `ws` replicas of the named
    workload (seeds 0 .. ws - 1, so the work per GPU stays that of one workload: weak scaling); its
    cells are split over the ranks by shard.partition_cells (LPT on 16 Q + 8 P^2 bytes), and each rank
    keeps its own cells of every replica.  At ws = 1 this is the workload itself."""
    if ws == 1:
        return _workload(args, seed=0, device=device)
    from paper_2606_21278_b300.shard import partition_cells
    reps = [_workload(args, seed=k, device=device) for k in range(ws)]
    counts = np.concatenate([r.counts().cpu().numpy() for r in reps])
    mine = partition_cells(counts, reps[0].modes, ws)[rank]
    base = np.cumsum([0] + [r.n_cells for r in reps])
    parts = []
    for k, r in enumerate(reps):
        sel = mine[(mine >= base[k]) & (mine < base[k + 1])] - base[k]
        parts.append(r.cell_slice(torch.as_tensor(sel, device=r.offsets.device)))
    cat = lambda f: torch.cat([getattr(q, f) for q in parts])
    offs = [torch.zeros(1, dtype=torch.int64, device=parts[0].offsets.device)]
    for q in parts:
        offs.append(q.offsets[1:] + offs[-1][-1])
    return synth.Workload(**{**parts[0].__dict__, "n_cells": int(sum(q.n_cells for q in parts)),
                             "nverts": cat("nverts"), "verts": cat("verts"), "offsets": torch.cat(offs),
                             "x": cat("x"), "y": cat("y"), "h": cat("h"), "w": cat("w")})


def _capture(fn):
    """CUDA graph of fn() (stream-ordered library calls only), warmed up on a side stream first."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


def _time_graph(g, steps, warmup=2):
    """Per-replay CUDA-event times (ms) of a captured graph on the current stream."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        a.record(stream)
        g.replay()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


REF_POOL = 4096   # cells the reference arm draws its steps from


def _config_cells(name):
    """Number of cells of a named workload."""
    spec = synth.CONFIGS[name]
    if spec["kind"] == "ico":
        return 20 * 4 ** spec["level"]
    if spec["kind"] == "mixed":
        return spec["n_tri"] + spec["n_hex"]
    return spec["n_cells"]


def run_reference(args):
    """The oracle (FP64 direct sums + EMS) on the host cores: every step is a bounded seeded sample
    of the workload's cells, sized from the warm-up so that the whole run takes about
    --ref-seconds."""
    import oracle
    ws, rank = _dist()
    if rank != 0:
        return
    oracle.lib()   # compile/load before anything is timed
    # a seeded pool of at most REF_POOL cells of the workload (the steps cycle through it): the host
    # never holds the whole batch, whose 5.6e8 samples of the 81,920-cell configuration would take
    # tens of GB and minutes to generate on the CPU
    full = _config_cells(args.workload)
    pool = argparse.Namespace(**{**vars(args), "cells": min(args.cells or full, full, REF_POOL)})
    wl = _workload(pool, seed=0, device="cpu")
    rng = np.random.default_rng(0)
    order = rng.permutation(wl.n_cells)
    # calibrate on as many cells as keep every host thread busy (warm-up); the steps below use at
    # least as many, so the oracle runs at its parallel rate rather than on one or two large cells
    busy = 4 * (os.cpu_count() or 1)
    n = max(1, min(busy, wl.n_cells))
    per_point = None
    pos = 0
    for _ in range(max(1, args.warmup)):
        sub = wl.cell_slice(sorted(order[pos:pos + n].tolist()))
        pos = (pos + n) % max(1, wl.n_cells - n)
        t0 = time.perf_counter()
        oracle.ems(oracle.type1(sub))
        per_point = (time.perf_counter() - t0) / max(1, sub.n_points)
    mean_q = wl.n_points / max(1, wl.n_cells)
    cells_per_step = int(max(min(busy, wl.n_cells), min(wl.n_cells, args.ref_seconds / max(1, args.steps) / (per_point * mean_q))))
    pts, secs = 0, 0.0
    for _ in range(args.steps):
        sub = wl.cell_slice(sorted(order[pos:pos + cells_per_step].tolist()))
        pos = (pos + cells_per_step) % max(1, wl.n_cells - cells_per_step)
        t0 = time.perf_counter()
        oracle.ems(oracle.type1(sub))
        secs += time.perf_counter() - t0
        pts += sub.n_points
    rate = pts / secs
    spec = synth.CONFIGS[args.workload]
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "points/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "modes": spec["modes"], "cells_per_step": cells_per_step},
            "cpu_baseline": {"value": rate, "unit": "points/s", "cores": oracle.threads_used(), "kind": "oracle",
                             "sample": f"{args.steps} steps of {cells_per_step} cells drawn from a seeded pool of "
                                       f"{wl.n_cells} cells of {args.workload} ({pts} points in total), "
                                       f"type-1 + EMS, FP64 direct sum"},
            "e2e": {"value": rate, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _bf16_peak():
    """Dense tensor-core peak (TFLOP/s) for a kernel timed on its own: the measured bf16 burst figure;
    binary16 operands run at the same nominal rate (2.25 PFLOP/s dense for both)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)).get("bf16_tflops", 1800.0), "measured (bf16 burst; f16 at the same nominal rate)"
    return 1800.0, "fallback"


def _alg_bytes(wl, P, k_max):
    """Algorithmic bytes of one type-1 + EMS pass: 16 B per sample in, 8 P^2 B of coefficients and
    4 + 4 K_max + 8 B of EMS results per cell out."""
    return 16 * wl.n_points + 8 * P * P * wl.n_cells + (4 + 4 * k_max + 8) * wl.n_cells


def _route_timings(enufft, wl, args, prm, steps):
    """Each execution route of the step on its own cells, in its own captured graph: the fused
    spread/FFT kernel on the cells above the tensor-core threshold, the tensor-core direct sum on the
    rest.  Returns a dict per route with its time and roofline (HBM bytes for the fused kernel; the
    method's 8 P^2 Q flops per cell against the tensor peak for the direct sum)."""
    P = wl.modes
    cnt = wl.counts()
    hbm, hbm_src = _peaks()
    tc_peak, tc_src = _bf16_peak()
    out = {}
    tc = int(wl.tc_max_points)
    groups = [("fused", torch.nonzero(cnt > tc).flatten() if tc > 0 else None, 0),
              ("tensor_core", torch.nonzero(cnt <= tc).flatten() if tc > 0 else None, tc)]
    for name, cells, thr in groups:
        if cells is None or len(cells) == 0:
            continue
        sub = wl.cell_slice(cells)
        plan = enufft.Plan.for_workload(sub, tc_max_points=(1 << 30) if thr else 0, kernel=args.kernel,
                                        frame=args.frame)
        co = plan.new_coeffs()
        o = plan._ems_out(prm)
        g = _capture(lambda: plan.type1_ems(sub.x, sub.y, sub.h, sub.w, prm, coeffs=co, out=o))
        ms = float(np.mean(_time_graph(g, steps)))
        plan.sync_status()
        ab = _alg_bytes(sub, P, prm.k_max)
        gbs = ab / (ms * 1e-3) / 1e9
        r = {"cells": sub.n_cells, "points": sub.n_points, "ms": ms, "points_per_s": sub.n_points / (ms * 1e-3),
             "hbm": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "peak_source": hbm_src,
                     "algorithmic_bytes_per_launch": ab}}
        if name == "tensor_core":
            fl = 8.0 * P * P * sub.n_points
            tf = fl / (ms * 1e-3) / 1e12
            exe = 3 * 2 * 128 * 80 * float(sub.n_points)   # three split products of 128 x 80 per sample
            r["tensor"] = {"achieved": tf, "peak": tc_peak, "unit": "TFLOP/s", "frac": tf / tc_peak,
                           "peak_source": tc_src, "flops_per_launch": fl,
                           "executed_tflops": exe / (ms * 1e-3) / 1e12,
                           "note": "method's work 8 P^2 Q; executed: three f16 products (hi hi, hi lo, lo hi) of the "
                                   "128 features of the modes n by the 80 of the modes m' = 0..P/2 per sample"}
        out[name] = r
        del g, plan, co, o, sub
    return out


def run_ours(args):
    import paper_2606_21278_b300 as enufft
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    wl = _rank_workload(args, ws, rank, "cuda")
    # n_f = 256 workloads take the subgrid tile the plan's tuner picks (16, 32 or 64 nodes), as their
    # configuration prescribes; the others keep their prescribed routes
    large = int(round(wl.sigma * wl.modes)) > 128
    plan = enufft.Plan.for_workload(wl, kernel=args.kernel, frame=args.frame, autotune=large,
                                    tune_cache=args.tune_cache if large else None)
    info = plan.info()
    prm = enufft.EMSParams()
    coeffs = plan.new_coeffs()
    ks, sel, ret = plan._ems_out(prm)
    stream = torch.cuda.current_stream()

    def step(x, y, h, w):
        plan.type1_ems(x, y, h, w, prm, coeffs=coeffs, out=(ks, sel, ret))

    # the step (every kernel of enufft_type1_ems) through the plan's own CUDA graph: captured by the
    # first call, replayed by every later one
    for _ in range(args.warmup):
        step(wl.x, wl.y, wl.h, wl.w)
    torch.cuda.synchronize()
    plan.sync_status()

    def graph_step():
        plan.type1_ems_graph(wl.x, wl.y, wl.h, wl.w, coeffs, (ks, sel, ret), prm)

    for _ in range(args.warmup):
        graph_step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    _barrier(ws)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            graph_step()
            ev[i][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
    _barrier(ws)
    plan.sync_status()
    total_ms = _max_over_ranks(t0.elapsed_time(t1), ws)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    ms = total_ms / args.steps
    pts_all = _sum_over_ranks(float(wl.n_points), ws)
    value = pts_all / (ms * 1e-3)
    P = wl.modes
    peak, peak_src = _peaks()
    tc_peak, _ = _bf16_peak()

    # each route on its own (the dominant kernel's roofline is taken from its own launches)
    routes = _route_timings(enufft, wl, args, prm, max(3, min(args.steps, 10))) if info["cells_large"] == 0 else {}
    alg_all = _alg_bytes(wl, P, prm.k_max)
    if info["cells_large"] == 0 and info["cells_tensor"] == 0:   # one route: the step itself
        kms = float(np.mean(launch_ms))
        gbs = alg_all / (kms * 1e-3) / 1e9
        routes["fused"] = {"cells": wl.n_cells, "points": wl.n_points, "ms": kms, "points_per_s": wl.n_points / (kms * 1e-3),
                           "hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                                   "peak_source": peak_src, "algorithmic_bytes_per_launch": alg_all}}
    if info["cells_large"]:
        kern = "n_f = 256 route, whole step (sort, scale, tile spread, FFT, EMS finish)"
        ach = alg_all / (float(np.mean(launch_ms)) * 1e-3) / 1e9
    else:
        fr = routes["fused"] if "fused" in routes else routes["tensor_core"]
        kern = (f"type1_fused_kernel<float,{info['fine_grid']},{info['kernel_width']}> (+ EMS finish"
                + (", local-coordinate pre-pass)" if args.frame == "edge" else ")")) if "fused" in routes \
            else "tc_nudft_kernel (+ EMS finish)"
        ach = fr["hbm"]["achieved"]
    roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": _traffic(args.workload) if args.frame == "centroid" else None, "peak_source": peak_src,
            "kernel": kern, "algorithmic_bytes_per_launch": routes["fused"]["hbm"]["algorithmic_bytes_per_launch"]
            if "fused" in routes else alg_all}
    # the fused kernel's other bounds: its algorithmic binary32 arithmetic against the FP32 peak, and
    # its w^2 shared-memory reductions per sample against the conflict-free reduction rate (both
    # measured by enufft_probe_peaks; the figures of the last probe are kept below)
    if "fused" in routes and info["cells_large"] == 0:
        fr = routes["fused"]
        Wd = info["kernel_width"]
        nf = info["fine_grid"]
        flops = (12 * Wd + Wd + 2 * Wd * Wd) * fr["points"] + \
            (2.5 * nf * nf * math.log2(nf * nf) + 2 * P * P + 4 * P * P // 2) * fr["cells"]
        t_hbm = fr["hbm"]["algorithmic_bytes_per_launch"] / (peak * 1e9)
        t_alu = flops / (FP32_TFLOPS * 1e12)
        t_red = Wd * Wd * fr["points"] / (SMEM_RED_GOPS * 1e9)
        t_bind = max(t_hbm, t_alu, t_red)
        fr["roofline_terms"] = {
            "hbm_ms": 1e3 * t_hbm, "alu_fp32_ms": 1e3 * t_alu, "smem_red_ms": 1e3 * t_red,
            "binding": ["hbm", "alu_fp32", "smem_red"][[t_hbm, t_alu, t_red].index(t_bind)],
            "frac_of_binding": 1e3 * t_bind / fr["ms"], "alu_flops_per_launch": flops,
            "alu_peak_tflops": FP32_TFLOPS, "smem_red_peak_gops": SMEM_RED_GOPS,
            "note": "alu: 12w (kernel values) + w + 2w^2 (taps) flops per sample, 2.5 n^2 log2 n^2 + 4P^2 per cell"}
    # the whole step against the batch roofline max(bytes / HBM, method flops / tensor peak)
    tc_flops = 8.0 * P * P * sum(int(c) for c in wl.counts()[wl.counts() <= wl.tc_max_points].tolist()) \
        if wl.tc_max_points > 0 else 0.0
    t_roof = max(alg_all / (peak * 1e9), tc_flops / (tc_peak * 1e12))
    step_roof = {"t_roof_ms": 1e3 * t_roof, "t_step_ms": ms, "frac": 1e3 * t_roof / ms,
                 "bound": "hbm" if alg_all / (peak * 1e9) >= tc_flops / (tc_peak * 1e12) else "tensor",
                 "algorithmic_bytes": alg_all, "tensor_flops": tc_flops}

    # the same step with the routes tuned at plan creation (threshold at most the workload's cap)
    tuned = None
    if not args.no_tune and wl.x.dtype == torch.float32:   # routes (fused / tensor core) or the n_f = 256 tile
        tplan = enufft.Plan.for_workload(wl, kernel=args.kernel, frame=args.frame, autotune=True)
        tinfo = tplan.info()
        tco = tplan.new_coeffs()
        tout = tplan._ems_out(prm)
        tg = _capture(lambda: tplan.type1_ems(wl.x, wl.y, wl.h, wl.w, prm, coeffs=tco, out=tout))
        tms = _max_over_ranks(float(np.mean(_time_graph(tg, max(3, min(args.steps, 10))))), ws)
        tplan.sync_status()
        tuned = {"ms_per_step": tms, "value": pts_all / (tms * 1e-3), "unit": "points/s",
                 "tuning": tplan.tuning(), "cells_tensor_core": tinfo["cells_tensor"],
                 "cells_fused": tinfo["cells_fused"], "large_tile": tinfo["large_tile"]}
        del tg, tplan, tco, tout

    # end to end through the public API with host buffers (pinned), copies inside the timed region:
    # step i's inputs go host -> device on a copy stream into one of two device buffer sets while
    # step i - 1 computes from the other (a streaming caller's double buffering), and every step's
    # EMS results come back to pinned host memory
    hx, hy, hh, hw = (t.cpu().pin_memory() for t in (wl.x, wl.y, wl.h, wl.w))
    dsets = [tuple(torch.empty_like(t) for t in (wl.x, wl.y, wl.h, wl.w)) for _ in range(2)]
    outs = [(coeffs, (ks, sel, ret)), (plan.new_coeffs(), plan.new_ems_out(prm))]
    hks = torch.empty(ks.shape, dtype=ks.dtype).pin_memory()
    hsel = torch.empty(sel.shape, dtype=sel.dtype).pin_memory()
    hret = torch.empty(ret.shape, dtype=ret.dtype).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    cstream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]
    for e in used:
        e.record(stream)

    def e2e_step(i):
        k = i % 2
        with torch.cuda.stream(cstream):
            cstream.wait_event(used[k])   # step i - 2 has read this buffer set
            for d, hsrc in zip(dsets[k], (hx, hy, hh, hw)):
                d.copy_(hsrc, non_blocking=True)
            copied[k].record(cstream)
        stream.wait_event(copied[k])
        co, (k1, s1, r1) = outs[k]
        plan.type1_ems(*dsets[k], prm, coeffs=co, out=(k1, s1, r1))
        used[k].record(stream)
        hks.copy_(k1, non_blocking=True)
        hsel.copy_(s1, non_blocking=True)
        hret.copy_(r1, non_blocking=True)

    e2e_step(0)
    e2e_step(1)
    torch.cuda.synchronize()
    _barrier(ws)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    cstream.wait_stream(stream)   # no copy of the timed steps starts before `a`
    for i in range(e2e_steps):
        e2e_step(i)
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = _max_over_ranks(a.elapsed_time(b), ws) / e2e_steps
    h2d = 4 * wl.x.element_size() * wl.n_points
    d2h = ks.numel() * 4 + sel.numel() * 4 + ret.numel() * 8
    del hx, hy, hh, hw, dsets, outs

    # untimed parity of the benchmarked spectra against the binary64 oracle on a seeded sample of
    # cells (the 16 largest, the largest and smallest of the tensor-core cells, the rest random):
    # coefficient rel-l2, the end-to-end EMS mode-set gate, and the EMS taken in the kernel's precision
    parity = None
    if rank == 0 and not args.no_check:
        import oracle
        graph_step()
        torch.cuda.synchronize()
        cnt = wl.counts().cpu()
        order = torch.argsort(cnt, descending=True).tolist()
        pick = set(order[:16])
        if wl.tc_max_points > 0:
            tcc = [c for c in order if cnt[c] <= wl.tc_max_points]
            pick.update(tcc[:8] + tcc[-4:])
        rng = np.random.default_rng(1)
        target = min(wl.n_cells, args.check_cells)
        for c in rng.permutation(wl.n_cells).tolist():
            if len(pick) >= target:
                break
            pick.add(c)
        cells = sorted(pick)
        sub = wl.cell_slice(cells).to("cpu")
        t_o = time.perf_counter()
        ref = oracle.type1(sub)
        t_o = time.perf_counter() - t_o
        got = coeffs[cells].cpu().numpy()
        rel = np.linalg.norm((got - ref).reshape(len(cells), -1), axis=1) / np.linalg.norm(ref.reshape(len(cells), -1), axis=1)
        gks, gsel = ks[cells].cpu().numpy(), sel[cells].cpu().numpy()
        gate = oracle.mode_set_gate(got, gks, gsel, ref, oracle.EMSParams())
        oks, osel, _, _ = oracle.ems(got, oracle.EMSParams(), energy_fp32=True)
        tc_in = int(sum(1 for c in cells if wl.tc_max_points and cnt[c] <= wl.tc_max_points))
        parity = {"cells": len(cells), "tensor_core_cells": tc_in, "points": sub.n_points,
                  "max_rel_l2": float(rel.max()), "median_rel_l2": float(np.median(rel)),
                  "ems_fp64_mismatches": len(gate["mismatches"]),
                  "ems_fp64_near_ties": sum(1 for m in gate["mismatches"] if m["near_tie"]),
                  "ems_identical": len(gate["mismatches"]) == 0,
                  "mismatches": gate["mismatches"][:8],
                  "ems_kernel_precision_identical": bool(np.array_equal(oks, gks) and np.array_equal(osel, gsel)),
                  "oracle_s": t_o}

    # Sec. 3.2 diagnostics on the benchmarked spectra and selection (reconstruction at every sample,
    # relative RMSE, Parseval variances), timed like the step; fused-route plans only
    recon = None
    if not args.no_reconstruct:
        hrec = torch.empty_like(wl.h)
        stats = torch.empty(wl.n_cells, 4, dtype=torch.float64, device="cuda")
        lib = enufft.load_library()
        import ctypes
        ptr = lambda t: ctypes.c_void_p(t.data_ptr())

        def rstep():
            lib.enufft_set_stream(plan._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            st = lib.enufft_reconstruct(plan._h, ptr(coeffs), ptr(ks), ptr(sel), prm.k_max, ptr(wl.x), ptr(wl.y),
                                        ptr(wl.h), ptr(wl.w), ptr(hrec), ptr(stats))
            if st != 0:
                raise RuntimeError(lib.enufft_last_error(plan._h).decode())

        rg = _capture(rstep)
        rsteps = max(3, min(args.steps, 20))
        rms = _max_over_ranks(float(np.mean(_time_graph(rg, rsteps))), ws)
        plan.sync_status()
        rbytes = 20 * wl.n_points + (8 * P * P + 4 + 4 * prm.k_max + 32) * wl.n_cells
        rach = rbytes / (rms * 1e-3) / 1e9
        recon = {"ms": rms, "value": pts_all / (rms * 1e-3), "unit": "points/s", "steps": rsteps,
                 "kernel": (f"type1_adjoint_kernel<float,{info['fine_grid']},{info['kernel_width']}> (reconstruction mode)"
                            if info["cells_large"] == 0 else
                            "large_adj_fft_kernel + large_interp_kernel + large_recon_stats_kernel (reconstruction mode)"),
                 "roofline": {"bound": "hbm", "achieved": rach, "peak": peak, "unit": "GB/s", "frac": rach / peak,
                              "algorithmic_bytes_per_launch": rbytes},
                 "median_eps_rel": float(stats[:, 0].median().item())}
        del rg, hrec, stats

    # Voronoi quadrature weights by raster sampling (App. A) for the workload's samples, ng = 64:
    # a once-per-mesh preprocessing step, timed for reference (binary32 plans of the fused route)
    voronoi = None
    if not args.no_voronoi and info["cells_large"] == 0 and wl.x.dtype == torch.float32 and args.frame == "centroid":
        ng = 64
        wv = torch.empty_like(wl.w)
        plan.voronoi_weights(wl.x, wl.y, ng)
        torch.cuda.synchronize()
        v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        vsteps = 3
        v0.record(stream)
        for _ in range(vsteps):
            wv = plan.voronoi_weights(wl.x, wl.y, ng)
        v1.record(stream)
        torch.cuda.synchronize()
        vms = _max_over_ranks(v0.elapsed_time(v1), ws) / vsteps
        plan.sync_status()
        searches = float(ng * ng) * wl.n_cells
        voronoi = {"ms": vms, "value": pts_all / (vms * 1e-3), "unit": "points/s", "steps": vsteps, "ng": ng,
                   "raster_searches_per_s": _sum_over_ranks(searches, ws) / (vms * 1e-3),
                   "kernel": "voronoi_kernel (bucketed nearest sample, certified binary32, binary64 near ties)"}
        del wv

    # the differentiation workload (4,096 hexagons, 48 x 48 modes): forward type-1 + EMS, loss L =
    # sum of the EMS-retained power over cells (one binary64 scalar all-reduced over the ranks, the
    # only collective), backward through the hand-written adjoint to dL/dh and dL/dw
    gradient = None
    if not args.no_gradient:
        gw_ = synth.make("hex4096_p48", seed=rank, device="cuda")
        gplan = enufft.Plan.for_workload(gw_)
        hh_ = gw_.h.clone().requires_grad_(True)
        ww_ = gw_.w.clone().requires_grad_(True)

        def gstep():
            hh_.grad = None
            ww_.grad = None
            power, _, _, _ = enufft.EMSRetainedPower.apply(hh_, ww_, gplan, gw_.x, gw_.y)
            L = power.sum()
            L.backward()
            return L

        for _ in range(3):
            gstep()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gsteps = max(3, min(args.steps, 10))
        g0.record(stream)
        for _ in range(gsteps):
            L = gstep()
        g1.record(stream)
        torch.cuda.synchronize()
        gms = _max_over_ranks(g0.elapsed_time(g1), ws) / gsteps
        gplan.sync_status()
        L_all = _sum_over_ranks(float(L.item()), ws)
        gpts = _sum_over_ranks(float(gw_.n_points), ws)
        gradient = {"workload": "hex4096_p48", "ms": gms, "value": gpts / (gms * 1e-3), "unit": "points/s",
                    "steps": gsteps, "loss": L_all,
                    "kernels": "type1_fused_kernel + ems_finish_kernel + ems_backward_kernel + type1_adjoint_kernel",
                    "collective": "one binary64 scalar all-reduce of L per step" if ws > 1 else "none (1 rank)"}
        del gplan, hh_, ww_, gw_

    # the plain binary32 per-cell path on the same workload (one launch sequence per cell), for the
    # speed-up the metric states; timed the same way, fewer steps
    plain = None
    if not args.no_plain:
        pplan = enufft.Plan.for_workload(wl, precision="fp32", tc_max_points=0, kernel=args.kernel,
                                         frame=args.frame)
        pco = pplan.new_coeffs()
        pout = pplan._ems_out(prm)

        def pstep():
            pplan.type1_ems(wl.x, wl.y, wl.h, wl.w, prm, coeffs=pco, out=pout)

        psteps = 3
        pstep()
        torch.cuda.synchronize()
        _barrier(ws)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(psteps):
            pstep()
        a1.record(stream)
        torch.cuda.synchronize()
        pms = _max_over_ranks(a0.elapsed_time(a1), ws) / psteps
        pplan.sync_status()
        plain = {"value": pts_all / (pms * 1e-3), "unit": "points/s", "ms_per_step": pms, "steps": psteps,
                 "speedup": pms / ms, "launches_per_step": pplan.info()["kernels_per_type1_ems"],
                 "note": "one launch sequence per cell (memset, spread, row FFT, column FFT, deconvolve) + EMS"}
        del pplan, pco, pout

    cpu_base = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, cells_s, pts_s, thr, dt = _oracle_sample(lambda: wl.to("cpu"), target_s=args.ref_seconds / 4)
        cpu_base = {"value": rate, "unit": "points/s", "cores": thr, "kind": "oracle",
                    "sample": f"{cells_s} seeded cells ({pts_s} points) of {args.workload}, type-1 + EMS, FP64 direct sum, {dt:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms,
                "step_ms": {"median": float(np.median(launch_ms)), "best": float(np.min(launch_ms)),
                            "mean": float(np.mean(launch_ms))},
                "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "n_cells": wl.n_cells, "n_points": wl.n_points, "modes": P,
                           "cells_fused": info["cells_fused"], "cells_tensor_core": info["cells_tensor"],
                           "cells_large": info["cells_large"], "tc_max_points": wl.tc_max_points,
                           **({"q_scale": args.q_scale} if args.q_scale != 1.0 else {}),
                           **({"max_q": args.max_q} if args.max_q is not None else {}),
                           **({"cells_subset": args.cells} if args.cells is not None else {}),
                           "fine_grid": info["fine_grid"], "kernel_width": info["kernel_width"],
                           "large_tile": info["large_tile"], **({"large_tile_from": "plan tuner"} if large else {}),
                           "kernel": args.kernel, "frame": args.frame, "precision": "mixed",
                           "ems": "K_max 12, alpha 0..0.7, delta 0.02, HEAD sums",
                           "timing": "one replay per step of the plan-owned CUDA graph of enufft_type1_ems (enufft_type1_ems_graph)",
                           "l2": f"inputs larger than L2 ({16 * wl.n_points / 1e9:.2f} GB of samples per step)",
                           "parallelism": (f"cells of {ws} seeded replicas split over {ws} ranks by LPT"
                                           if ws > 1 else "1 rank")},
                "roofline": roof, "routes": routes, "step_roofline": step_roof, "cpu_baseline": cpu_base,
                "e2e": {"value": pts_all / (e2e_ms * 1e-3), "unit": "points/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                        "pipeline": "step i + 1's host-to-device copy (copy stream) overlaps step i's compute; "
                                    "two device input sets; enufft_type1_ems per step"},
                "tuned_routes": tuned,
                "plain_fp32": plain,
                "reconstruct": recon,
                "voronoi": voronoi,
                "gradient": gradient,
                "gpu_launches": info["kernels_per_type1_ems"] * args.steps,
                "clocks": clk.summary(), "parity": parity}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_error_vs_width(args):
    """Accuracy of the transform against the oracle as a function of the kernel width w on the single
    equilateral triangle (2000 samples, P = 32, sigma = 2): binary32 (mixed) plans for w = 4..10 and
    binary64 plans for w = 8..13, with tol = 0 so that w is used as given, for the ES and the KB
    kernel.  One JSON line."""
    import oracle
    import paper_2606_21278_b300 as enufft
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    wl64 = synth.make("tri1_q2000_p32_fp64", seed=0)
    ref = oracle.type1(wl64)
    rows = []
    for kernel in ("es", "kb"):
        for prec, widths in (("mixed", range(4, 11)), ("fp64", range(8, 14))):
            wl = wl64 if prec == "fp64" else synth.Workload(**{**wl64.__dict__, **{
                k: getattr(wl64, k).float() for k in ("x", "y", "h", "w")}})
            g = wl.to("cuda")
            for wd in widths:
                plan = enufft.Plan.for_workload(g, kernel_width=wd, tol=0.0, precision=prec, kernel=kernel)
                c = plan.type1(g.x, g.y, g.h, g.w)
                plan.sync_status()
                cn = c.cpu().numpy().astype(np.complex128)
                rows.append({"kernel": kernel, "precision": prec, "w": wd, "fine_grid": plan.info()["fine_grid"],
                             "rel_l2": float(np.linalg.norm(cn - ref) / np.linalg.norm(ref))})
    print(json.dumps({"error_vs_width": rows, "workload": "tri1_q2000_p32_fp64", "modes": 32, "sigma": 2.0}),
          flush=True)


def run_mono_sweep(args):
    """The monochromatic sweep of Sec. 3.1 (Table mono_sweep_config) on the GPU: for every expansion
    ratio, window mask (triangle, square, circle) and weighting (uniform, Voronoi), the type-1
    transform of all (dy, theta, u, Q) cells (P = 16, KB kernel) and EMS at every K_max; per cell
    the recovered peak pair's direction error (degrees, modulo 180) and amplitude error against
    A / 2, and K* / K_max.  Prints pooled median and standard deviation per sweep value and mask.
    The oversampling axis leaves n_f = 64 for P = 16 (the smallest fine grid), so its rows repeat."""
    import paper_2606_21278_b300 as enufft
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    A, P = 1000.0, 16
    rows = {mk: [] for mk in ("triangle", "square", "circle")}
    gpu_ms = 0.0
    for r_exp in synth.MONO_AXES["r_exp"]:
        wl, meta = synth.mono_sweep(r_exp, amplitude=A, modes=P)
        g = wl.to("cuda")
        for mk, mask in (("triangle", 0), ("square", 1), ("circle", 2)):
            plan = enufft.Plan(g.offsets, g.nverts, g.verts, modes=P, oversamp=2.0, kernel_width=7, tol=1e-6,
                               precision="mixed", mask=mask, eta=r_exp, kernel="kb")
            for wname in ("uniform", "voronoi"):
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record()
                w = g.w if wname == "uniform" else plan.voronoi_weights(g.x, g.y, 64)
                c = plan.type1(g.x, g.y, g.h, w)
                outs = [plan.ems(c, enufft.EMSParams(k_max=K)) for K in synth.MONO_AXES["k_max"]]
                a1.record()
                torch.cuda.synchronize()
                gpu_ms += a0.elapsed_time(a1)
                plan.sync_status()
                cn = c.cpu().numpy()
                for K, (ks, sel, _) in zip(synth.MONO_AXES["k_max"], outs):
                    ks, sel = ks.cpu().numpy(), sel.cpu().numpy()
                    for j in range(wl.n_cells):
                        if ks[j] < 1:
                            continue
                        p = int(sel[j, 0])
                        m, n = p % P - P // 2, p // P - P // 2
                        tr = math.degrees(math.atan2(n, m)) % 180.0
                        tt = math.degrees(math.atan2(meta["n"][j], meta["m"][j])) % 180.0
                        d = abs(tr - tt)
                        rows[mk].append(dict(dy=meta["dy"][j], theta=meta["theta"][j], u=meta["u"][j],
                                             r_exp=r_exp, Q=meta["Q"][j], k_max=K, weights=wname,
                                             dtheta=min(d, 180.0 - d),
                                             dA=abs(abs(cn[j, n + P // 2, m + P // 2]) - A / 2),
                                             budget=ks[j] / K))
    table = {}
    for mk, rs in rows.items():
        t = {}
        for ax in ("theta", "dy", "u", "r_exp", "Q", "k_max", "weights"):
            t[ax] = {}
            for v in sorted({r[ax] for r in rs}, key=str):
                sub = [r for r in rs if r[ax] == v]
                t[ax][str(v)] = {q: [float(np.median([r[q] for r in sub])), float(np.std([r[q] for r in sub]))]
                                 for q in ("dtheta", "dA", "budget")}
        t["all"] = {q: [float(np.median([r[q] for r in rs])), float(np.std([r[q] for r in rs]))]
                    for q in ("dtheta", "dA", "budget")}
        table[mk] = t
    print(json.dumps({"mono_sweep": table, "rows_per_mask": {k: len(v) for k, v in rows.items()},
                      "gpu_ms": gpu_ms, "modes": P, "amplitude": A, "kernel": "kb",
                      "sigma_axis": "no effect: n_f = 64 for every sigma at P = 16"}), flush=True)


def run_peaks(args):
    """The GPU's measured compute peaks (enufft_probe_peaks) and the copy/bf16 peaks of the peaks
    file, as one JSON line."""
    import paper_2606_21278_b300 as enufft
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        pk = enufft.probe_peaks()
    print(json.dumps({"peaks": pk, "hbm_gbs": _peaks()[0], "bf16_tflops": _bf16_peak()[0],
                      "gpu": torch.cuda.get_device_name(), "clocks": clk.summary()}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=list(synth.CONFIGS))
    ap.add_argument("--cells", type=int, default=None, help="seeded subset of cells (profiling runs)")
    ap.add_argument("--q-scale", type=float, default=1.0, help="scale of the per-cell sample counts")
    ap.add_argument("--max-q", type=int, default=None, help="cap every cell at this many samples")
    ap.add_argument("--tc-max-points", type=int, default=None,
                    help="override the tensor-core routing threshold (cells with at most this many samples)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="CPU seconds of the reference arm (and a quarter of it for the cpu_baseline sample)")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain FP32 per-cell path")
    ap.add_argument("--no-reconstruct", action="store_true", help="skip timing the reconstruction diagnostics")
    ap.add_argument("--no-voronoi", action="store_true", help="skip timing the Voronoi quadrature weights")
    ap.add_argument("--no-gradient", action="store_true", help="skip timing the differentiation workload")
    ap.add_argument("--no-tune", action="store_true", help="skip timing the step with tuned routes")
    ap.add_argument("--tune-cache", default=None,
                    help="route-tuning cache file for the n_f = 256 tile choice (a second run reads it, no trial launches)")
    ap.add_argument("--check-cells", type=int, default=1024,
                    help="cells of the untimed parity check against the binary64 oracle")
    ap.add_argument("--kernel", default="es", choices=["es", "kb"],
                    help="spreading kernel: exponential of semicircle (default) or Kaiser-Bessel")
    ap.add_argument("--frame", default="centroid", choices=["centroid", "edge"],
                    help="local frame of every cell: centroid-aligned (default) or edge-aligned")
    ap.add_argument("--error-vs-width", action="store_true",
                    help="print the rel-l2 error against the oracle for kernel widths 4..13 (single triangle) and exit")
    ap.add_argument("--peaks", action="store_true", help="measure the GPU's compute peaks and exit")
    ap.add_argument("--mono-sweep", action="store_true", help="run the monochromatic sweep (Sec. 3.1) and exit")
    args = ap.parse_args()
    if args.peaks:
        run_peaks(args)
    elif args.mono_sweep:
        run_mono_sweep(args)
    elif args.error_vs_width:
        run_error_vs_width(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
