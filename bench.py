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
DEFAULT_WORKLOAD = "tri20480_p64"
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


def run_reference(args):
    """The oracle (FP64 direct sums + EMS) on the host cores: every step is a bounded seeded sample
    of the workload's cells, sized from the warm-up so that the whole run takes about
    --ref-seconds."""
    import oracle
    ws, rank = _dist()
    if rank != 0:
        return
    oracle.lib()   # compile/load before anything is timed
    wl = _workload(args, seed=0, device="cpu")
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
                             "sample": f"{args.steps} steps of {cells_per_step} seeded cells of {args.workload} "
                                       f"({pts} points in total), type-1 + EMS, FP64 direct sum"},
            "e2e": {"value": rate, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import paper_2606_21278_b300 as enufft
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    wl = _workload(args, seed=rank, device="cuda")
    plan = enufft.Plan.for_workload(wl, kernel=args.kernel, frame=args.frame)
    info = plan.info()
    prm = enufft.EMSParams()
    coeffs = plan.new_coeffs()
    ks = torch.empty(wl.n_cells, dtype=torch.int32, device="cuda")
    sel = torch.empty(wl.n_cells, prm.k_max, dtype=torch.int32, device="cuda")
    ret = torch.empty(wl.n_cells, dtype=torch.float64, device="cuda")
    import ctypes
    lib = enufft.load_library()
    pc = prm.c()
    stream = torch.cuda.current_stream()
    lib.enufft_set_stream(plan._h, ctypes.c_void_p(stream.cuda_stream))
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())

    def step(x, y, h, w):
        st = lib.enufft_type1_ems(plan._h, ptr(x), ptr(y), ptr(h), ptr(w), ptr(coeffs), None, 0, ctypes.byref(pc),
                                  ptr(ks), ptr(sel), ptr(ret))
        if st != 0:
            raise RuntimeError(lib.enufft_last_error(plan._h).decode())

    for _ in range(args.warmup):
        step(wl.x, wl.y, wl.h, wl.w)
    torch.cuda.synchronize()
    plan.sync_status()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    _barrier(ws)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            step(wl.x, wl.y, wl.h, wl.w)
            ev[i][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    _barrier(ws)
    total_ms = _max_over_ranks(t0.elapsed_time(t1), ws)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    ms = total_ms / args.steps
    pts_all = _sum_over_ranks(float(wl.n_points), ws)
    value = pts_all / (ms * 1e-3)

    # roofline of the dominant kernel (the fused type-1 + EMS kernel is the only kernel of the step)
    P = wl.modes
    alg_bytes = 16 * wl.n_points + 8 * P * P * wl.n_cells + (4 + 4 * prm.k_max + 8) * wl.n_cells
    kern_ms = float(np.mean(launch_ms))
    peak, peak_src = _peaks()
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": _traffic(args.workload) if args.frame == "centroid" else None, "peak_source": peak_src,
            "kernel": (f"type1_fused_kernel<float,{info['fine_grid']},{info['kernel_width']}> (+ EMS finish"
                       + (", local-coordinate pre-pass)" if args.frame == "edge" else ")") if info["cells_fused"]
                                  else "n_f = 256 route, whole step (sort, scale, tile spread, FFT, EMS finish)"),
            "algorithmic_bytes_per_launch": alg_bytes}

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    hx, hy, hh, hw = (t.cpu().pin_memory() for t in (wl.x, wl.y, wl.h, wl.w))
    dx, dy, dh, dw = (torch.empty_like(t) for t in (wl.x, wl.y, wl.h, wl.w))
    hks = torch.empty(ks.shape, dtype=ks.dtype).pin_memory()
    hsel = torch.empty(sel.shape, dtype=sel.dtype).pin_memory()
    hret = torch.empty(ret.shape, dtype=ret.dtype).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))

    def e2e_step():
        for d, hsrc in ((dx, hx), (dy, hy), (dh, hh), (dw, hw)):
            d.copy_(hsrc, non_blocking=True)
        step(dx, dy, dh, dw)
        hks.copy_(ks, non_blocking=True)
        hsel.copy_(sel, non_blocking=True)
        hret.copy_(ret, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    _barrier(ws)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = _max_over_ranks(a.elapsed_time(b), ws) / e2e_steps
    h2d = 4 * wl.x.element_size() * wl.n_points
    d2h = ks.numel() * 4 + sel.numel() * 4 + ret.numel() * 8

    # sampled parity of the benchmarked run against the oracle (a few cells; CPU, untimed)
    parity = None
    if rank == 0 and not args.no_check:
        import oracle
        step(wl.x, wl.y, wl.h, wl.w)
        torch.cuda.synchronize()
        cnt = wl.counts().cpu()
        cells = sorted(set(torch.argsort(cnt, descending=True)[:2].tolist() + [0, wl.n_cells // 2, wl.n_cells - 1]))
        sub = wl.cell_slice(cells).to("cpu")
        ref = oracle.type1(sub)
        got = coeffs[cells].cpu().numpy()
        rel = np.linalg.norm((got - ref).reshape(len(cells), -1), axis=1) / np.linalg.norm(ref.reshape(len(cells), -1), axis=1)
        oks, osel, _, _ = oracle.ems(got, oracle.EMSParams(), energy_fp32=True)
        parity = {"cells": len(cells), "max_rel_l2": float(rel.max()),
                  "ems_identical": bool(np.array_equal(oks, ks[cells].cpu().numpy()) and
                                        np.array_equal(osel, sel[cells].cpu().numpy()))}

    # Sec. 3.2 diagnostics on the benchmarked spectra and selection (reconstruction at every sample,
    # relative RMSE, Parseval variances), timed like the step; fused-route plans only
    recon = None
    if not args.no_reconstruct and info["cells_large"] == 0:
        hrec = torch.empty_like(wl.h)
        stats = torch.empty(wl.n_cells, 4, dtype=torch.float64, device="cuda")

        def rstep():
            st = lib.enufft_reconstruct(plan._h, ptr(coeffs), ptr(ks), ptr(sel), prm.k_max, ptr(wl.x), ptr(wl.y),
                                        ptr(wl.h), ptr(wl.w), ptr(hrec), ptr(stats))
            if st != 0:
                raise RuntimeError(lib.enufft_last_error(plan._h).decode())

        for _ in range(3):
            rstep()
        torch.cuda.synchronize()
        _barrier(ws)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        rsteps = max(3, min(args.steps, 20))
        r0.record(stream)
        for _ in range(rsteps):
            rstep()
        r1.record(stream)
        torch.cuda.synchronize()
        rms = _max_over_ranks(r0.elapsed_time(r1), ws) / rsteps
        plan.sync_status()
        rbytes = 20 * wl.n_points + (8 * P * P + 4 + 4 * prm.k_max + 32) * wl.n_cells
        rach = rbytes / (rms * 1e-3) / 1e9
        recon = {"ms": rms, "value": pts_all / (rms * 1e-3), "unit": "points/s", "steps": rsteps,
                 "kernel": f"type1_adjoint_kernel<float,{info['fine_grid']},{info['kernel_width']}> (reconstruction mode)",
                 "roofline": {"bound": "hbm", "achieved": rach, "peak": peak, "unit": "GB/s", "frac": rach / peak,
                              "algorithmic_bytes_per_launch": rbytes},
                 "median_eps_rel": float(stats[:, 0].median().item())}

    # Voronoi quadrature weights by raster sampling (App. A) for the workload's samples, ng = 64:
    # nearest windowed sample of every raster point (bucketed search); binary32 plans of the fused
    # route only (cells of more than 16384 samples fall back to a brute-force search)
    voronoi = None
    if not args.no_voronoi and info["cells_large"] == 0 and wl.x.dtype == torch.float32:
        ng = 64
        wv = torch.empty_like(wl.w)

        def vstep():
            st = lib.enufft_voronoi_weights(plan._h, ptr(wl.x), ptr(wl.y), ng, ptr(wv))
            if st != 0:
                raise RuntimeError(lib.enufft_last_error(plan._h).decode())

        vstep()
        torch.cuda.synchronize()
        _barrier(ws)
        v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        vsteps = 3
        v0.record(stream)
        for _ in range(vsteps):
            vstep()
        v1.record(stream)
        torch.cuda.synchronize()
        vms = _max_over_ranks(v0.elapsed_time(v1), ws) / vsteps
        plan.sync_status()
        searches = float(ng * ng) * wl.n_cells
        voronoi = {"ms": vms, "value": pts_all / (vms * 1e-3), "unit": "points/s", "steps": vsteps, "ng": ng,
                   "raster_searches_per_s": _sum_over_ranks(searches, ws) / (vms * 1e-3),
                   "kernel": "voronoi_kernel (bucketed nearest sample, binary32)"}

    # the plain binary32 per-cell path on the same workload (one launch sequence per cell), for the
    # speed-up the metric states; timed the same way, fewer steps
    plain = None
    if not args.no_plain:
        pplan = enufft.Plan.for_workload(wl, precision="fp32", tc_max_points=0, kernel=args.kernel,
                                         frame=args.frame)
        pco = pplan.new_coeffs()
        lib.enufft_set_stream(pplan._h, ctypes.c_void_p(stream.cuda_stream))

        def pstep():
            st = lib.enufft_type1_ems(pplan._h, ptr(wl.x), ptr(wl.y), ptr(wl.h), ptr(wl.w), ptr(pco), None, 0,
                                      ctypes.byref(pc), ptr(ks), ptr(sel), ptr(ret))
            if st != 0:
                raise RuntimeError(lib.enufft_last_error(pplan._h).decode())

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
                 "speedup": (pts_all / (ms * 1e-3)) / (pts_all / (pms * 1e-3)),
                 "launches_per_step": pplan.info()["kernels_per_type1_ems"]}
        del pplan, pco

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
                           "cells_tensor_core": info["cells_tensor"], "tc_max_points": wl.tc_max_points,
                           **({"q_scale": args.q_scale} if args.q_scale != 1.0 else {}),
                           **({"max_q": args.max_q} if args.max_q is not None else {}),
                           "fine_grid": info["fine_grid"], "kernel_width": info["kernel_width"],
                           "kernel": args.kernel, "frame": args.frame, "precision": "mixed", "ems": "K_max 12, alpha 0..0.7, delta 0.02, HEAD sums",
                           "l2": f"inputs larger than L2 ({16 * wl.n_points / 1e9:.2f} GB of samples per step)",
                           "parallelism": f"cells sharded, {ws} rank(s)"},
                "roofline": roof, "cpu_baseline": cpu_base,
                "e2e": {"value": pts_all / (e2e_ms * 1e-3), "unit": "points/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "plain_fp32": plain,
                "reconstruct": recon,
                "voronoi": voronoi,
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
    ap.add_argument("--kernel", default="es", choices=["es", "kb"],
                    help="spreading kernel: exponential of semicircle (default) or Kaiser-Bessel")
    ap.add_argument("--frame", default="centroid", choices=["centroid", "edge"],
                    help="local frame of every cell: centroid-aligned (default) or edge-aligned")
    ap.add_argument("--error-vs-width", action="store_true",
                    help="print the rel-l2 error against the oracle for kernel widths 4..13 (single triangle) and exit")
    args = ap.parse_args()
    if args.error_vs_width:
        run_error_vs_width(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
