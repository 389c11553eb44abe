"""Benchmark: voxel-iterations/s of the filtered-property FFT homogenisation hot path on GB300.

Workload (one "step"): the 2D resolution sweep of the centred-disk cell -- grids 45, 135, 405
and 1215 per side, contrasts 10 and 0.1, no filter / Voigt / Reuss / 2-layer filters (radius 1
pixel, 16x16 subgrid), 3 unit Mandel load cases -- i.e. 32 cells x 3 loads.  A step runs the
whole path: filter build (classification, subgrid sampling, homogenisation rule), the
fixed-point solve of every cell and load to convergence, and C_eff.  The FP32 form batches all
96 (cell, load) problems in one launch sequence (FP32 fields and FFTs, FP64 reductions); the
FP64 plain form solves one cell at a time in FP64.  Both stop on e_n < 1e-6.

value = sum over (cell, load) of n^2 * iterations, divided by the step time (FP32 batched).
Inputs are synthetic (seeded geometry; no dataset).  The working set (~1.8 GB of state) is
larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import hom_inputs as H  # noqa: E402

SIZES = (45, 135, 405, 1215)
CONTRASTS = (10.0, 0.1)
RULES = (H.RULE_NONE, H.RULE_VOIGT, H.RULE_REUSS, H.RULE_TWO_LAYER)
TOL = 1e-6
MAX_ITER = 3000
ENSEMBLE_MAX_ITER = 1000  # above ln(1e-6) / ln(99 / 101) ~ 690 iterations of the contrast-100 cells
METRIC = "voxel-iterations/s (2D resolution sweep, FP32 batched, e_n < 1e-6)"
UNIT = "voxel-it/s"


def workload():
    cells, phases = H.resolution_sweep_cells(SIZES, CONTRASTS, RULES, vf=0.2, radius_px=1.0, subgrid=16)
    c0 = []
    for cell in cells:
        pair = phases[cell.matrix_phase:cell.matrix_phase + 2]
        c0.append(H.mean_lame(pair))
    return cells, phases, np.array(c0)


def config_dict(extra=None):
    d = {"workload": "2D centred-disk resolution sweep: n in %s, contrasts %s, filters none/Voigt/Reuss/2-layer "
                     "(r = 1 px, S = 16), 3 Mandel unit loads, 32 cells x 3 loads per step" % (list(SIZES), list(CONTRASTS)),
         "tolerance": "e_n < %g" % TOL, "l2": "working set > L2 (no flush needed)"}
    if extra:
        d.update(extra)
    return d


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.stop = threading.Event()
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            if self.stop.is_set():
                break
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        self.stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for name, v in zip(names, r[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# DRAM bytes (read + write) per algorithmic byte of the specialised FP32 2D passes, from the ncu
# --set full capture of the profile case (--profile-case: two 1215^2 cells x 3 loads; traffic grows
# with the tiles processed, so a launch's traffic is this ratio times its bytes).
# Valid for the kernels as captured there; None for kernels without a capture.
TRAFFIC_RATIO = {"row": (110.233 + 52.886) / 215.77, "green": (177.580 + 116.155) / 354.61}


def golden_ceff():
    p = os.path.join(ROOT, "tests", "golden", "sweep2d_ceff.json")
    if not os.path.exists(p):
        return {}
    return {(e["n"], e["contrast"], e["rule"]): np.array(e["ceff"]) for e in json.load(open(p))["cells"]}


def ceff_errors(cells, phases, mean_sigma, gold):
    import paper_1412_3228_gb300 as hom
    C = hom.hom_effective_stiffness(np.eye(3), mean_sigma, 2)
    errs = []
    for i, cell in enumerate(cells):
        contrast = round(phases[cell.matrix_phase + 1][1] / phases[cell.matrix_phase][1], 6)
        key = (cell.n, contrast, H.RULE_NAMES[cell.rule])
        if key in gold:
            g = gold[key]
            errs.append(float(np.abs(C[i] - g).max() / np.abs(g).max()))
    return (max(errs) if errs else None), len(errs)


def reduce_across_ranks(ms: float, vox_it: float, device, world: int):
    """Job time = the slowest rank's timed region; work = the sum of every rank's voxel-iterations
    (each rank solves its own replica of the workload: weak scaling, no exchange on the data path)."""
    if world <= 1:
        return float(ms), float(vox_it)
    import torch
    ms_t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    vi_t = torch.tensor([float(vox_it)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(ms_t, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(vi_t, op=torch.distributed.ReduceOp.SUM)
    return float(ms_t.item()), float(vi_t.item())


def run_ours(args, rank, world):
    # the oracle's worker pool for the all-core CPU baseline, spawned before the first GPU call
    pool = None
    if rank == 0 and not args.skip_cpu:
        import multiprocessing as mp
        pool = mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1))
    import torch

    import paper_1412_3228_gb300 as hom
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cells, phases, c0 = workload()
    E = np.eye(3)
    stream = torch.cuda.current_stream()

    def step(stats=False, precision=hom.HOM_FP32, host_fields=False, fields=False, subset=None, production=False):
        # production: the whole solve as one graph launch with the autotuned plan (no per-kernel events)
        cs = cells if subset is None else [cells[i] for i in subset]
        cc = c0 if subset is None else c0[subset]
        mat = hom.hom_filter_build(cs, phases)
        r = hom.hom_solve(mat, E, cc, precision=precision, criterion=hom.HOM_CRIT_EN, tol=TOL, max_iter=MAX_ITER,
                          fields=fields, host_fields=host_fields, stats=stats, use_graph=production, tune=production)
        C = hom.hom_effective_stiffness(E, r["mean_sigma"], 2)
        return r, C

    for _ in range(args.warmup):
        step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # ---- timed region: K steps of the FP32 batched form, per-kernel events on the launch stream
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    vox_it = 0.0
    kstats = {}
    launches = 0
    with ClockSampler(dev.index) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            r, C = step(stats=True)
            vox_it += float(np.sum([[c.n ** 2 * it for it in r["iterations"][i]] for i, c in enumerate(cells)]))
            for k, v in r["stats"].items():
                s = kstats.setdefault(k, dict(launches=0, ms=0.0, bytes=0.0))
                s["launches"] += v["launches"]
                s["ms"] += v["ms"]
                s["bytes"] += v["bytes"]
            launches += sum(v["launches"] for v in r["stats"].values()) + 1  # + the filter-build kernel
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = t0.elapsed_time(t1)
    ms_max, vi_total = reduce_across_ranks(ms, vox_it, dev, world)
    value = vi_total / (ms_max / 1e3)
    fp32_err, ncmp = ceff_errors(cells, phases, r["mean_sigma"], golden_ceff())
    iters = r["iterations"]

    # ---- the filter build alone (part of every step above)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(3):
        hom.hom_filter_build(cells, phases)
    f1.record(stream)
    torch.cuda.synchronize()
    filter_ms = f0.elapsed_time(f1) / 3

    # ---- end to end: the public API with host outputs (fields and C_eff back on the host); the
    # warm-up steps let the pinned host buffers be allocated once and reused, as a caller would
    e2e_ms, e2e_vi, d2h = 0.0, 0.0, 0
    re_ = None
    for _ in range(max(2, args.warmup)):  # hold each result as the timed loop does: two buffer sets
        re_, Ce = step(host_fields=True, fields=True, production=True)
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(max(1, args.steps)):
        re_, Ce = step(host_fields=True, fields=True, production=True)
        e2e_vi += float(np.sum([[c.n ** 2 * it for it in re_["iterations"][i]] for i, c in enumerate(cells)]))
        d2h = (re_["eps"].numel() + re_["sigma"].numel()) * re_["eps"].element_size() + re_["mean_sigma"].nbytes + \
            re_["iterations"].nbytes * 2 + re_["err"].nbytes * 2
    torch.cuda.synchronize()
    e2e_total_s = time.perf_counter() - te
    e2e_ms = e2e_total_s * 1e3 / max(1, args.steps)
    h2d = sum(48 * len(c.prims) + 40 for c in cells) + 16 * len(phases) + 8 * E.size + 16 * len(cells)

    # ---- FP64 plain form: one cell at a time and batched, FP64 everywhere, against the FP32 form at
    # the same C_eff error (one untimed warm-up pass first)
    fp64 = None
    field_err = None
    if not args.skip_fp64 and rank == 0:
        fp64 = fp64_forms(hom, step, cells, phases, fp32_err)
        field_err = fp32_field_errors(hom, cells, phases, c0)
    # ---- comparison (not on the product path): cuFFT via torch.fft, a forward real 2D FFT and its
    # inverse over the 18 real fields of two 1215^2 cells x 3 loads x 3 components, against one
    # iteration of this library on the same cells (row pass + Green pass + control, CUDA events)
    comparison = None
    if rank == 0 and not args.skip_cufft:
        comparison = cufft_comparison(hom, cells, phases, c0, dev)

    # ---- secondary workloads: random-sphere cells (2-layer filter, 6 loads, FP32, e_n < 1e-6): 135^3
    # at both contrasts (C_eff against the oracle's stored values) and 243^3 at contrast 10
    spheres = spheres135 = None
    if rank == 0 and not args.skip_3d:
        spheres135 = spheres_3d(hom, dev, n=135, contrasts=(10.0, 0.1))
        spheres = spheres_3d(hom, dev, n=243, contrasts=(10.0,), fp64_check=not args.skip_fp64)

    # ---- secondary workload: the batched 2D ensemble (256 random-disk cells of uneven size)
    ensemble = None
    if rank == 0 and not args.skip_ensemble:
        ensemble = ensemble_2d(hom, dev)

    # ---- differentiation: FP32 forward + adjoint at 135^3 (von Mises + C_eff loss)
    backward = None
    if rank == 0 and not args.skip_3d:
        backward = backward_135(hom, dev)

    # ---- accelerated scheme (conjugate gradients) against the basic scheme at high contrast
    cg = None
    if rank == 0 and not args.skip_cg:
        cg = cg_comparison(hom, dev)

    # ---- the Eyre-Milton scheme on the sweep itself: time to solution against the basic scheme
    em_sweep = None
    if rank == 0 and not args.skip_cg:
        em_sweep = eyre_milton_sweep(hom, cells, phases, c0, fp32_err)

    # ---- roofline of the dominant kernel (largest share of kernel time)
    peak, peak_kind = measured_peak_hbm()
    dom = max((k for k in kstats if k in ("row", "green", "yfwd", "yinv")), key=lambda k: kstats[k]["ms"])
    ach = kstats[dom]["bytes"] / (kstats[dom]["ms"] / 1e3) / 1e9
    total_kms = sum(v["ms"] for v in kstats.values())
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "peak_source": peak_kind,
                "traffic": (round(TRAFFIC_RATIO[dom] * kstats[dom]["bytes"] / max(1, kstats[dom]["launches"]))
                            if dom in TRAFFIC_RATIO else None),
                "traffic_source": "ncu capture of two 1215^2 cells scaled to the launch's bytes",
                "bytes_per_launch": kstats[dom]["bytes"] / max(1, kstats[dom]["launches"]),
                "kernel_share": {k: round(v["ms"] / total_kms, 4) for k, v in kstats.items() if v["ms"] > 0},
                "achieved_gbs": {k: round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) for k, v in kstats.items()
                                 if v["ms"] > 0 and v["bytes"] > 0}}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 reductions)", "data": "synthetic",
            "config": config_dict({"parallelism": "replicas x%d (independent cells per rank)" % world,
                                   "cells": len(cells), "loads": 3}),
            "e2e": {"value": e2e_vi / e2e_total_s, "unit": UNIT, "ms_per_step": e2e_ms, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h),
                    "form": "public API, fields and C_eff to pinned host memory; whole solve as one graph launch, "
                            "autotuned plan"},
            "autotune": hom.hom_autotune_report().strip().splitlines(),
            "gpu_launches": launches, "roofline": roofline, "clocks": clk.summary(),
            "iterations": {"max": int(iters.max()), "min": int(iters.min()),
                           "per_rule": {H.RULE_NAMES[rr]: int(np.mean([iters[i].mean() for i, c in enumerate(cells)
                                                                        if c.rule == rr])) for rr in RULES}},
            "filter_build_ms": round(filter_ms, 3),
            "ceff_max_rel_err_vs_oracle": fp32_err, "ceff_cells_compared": ncmp,
            "fp32_field_errors": field_err,
            "fp64_plain": fp64,
            "fp32_vs_fp64_equal_error": (None if fp64 is None else {
                "fp32_value": value, "fp64_value": fp64["batched_equal_error"]["value"],
                "fp64_tol": fp64["batched_equal_error"]["tol"], "ratio": value / fp64["batched_equal_error"]["value"],
                "fp32_ceff_err": fp32_err, "fp64_ceff_err": fp64["batched_equal_error"]["ceff_max_rel_err"]}), "cufft_comparison": comparison, "spheres3d_243": spheres, "spheres3d_135": spheres135, "backward_135": backward,
            "ensemble2d_256": ensemble, "cg_vs_fixed_point": cg, "eyre_milton_sweep": em_sweep}
    if rank == 0 and not args.skip_cpu:
        line["cpu_baseline"] = cpu_baseline(args, pool)
    if pool is not None:
        pool.close()
        pool.join()
    return line


def flops_per_voxel_iteration(n, dim=2):
    """Algorithmic FLOPs of one voxel-iteration of one load (model): a forward and an inverse real
    FFT of each of the nc components (2 x 2.5 log2(N_v) each), the constitutive update (2 nc^2) and
    the Green operator with the residual (about 30 per voxel)."""
    nc = 3 if dim == 2 else 6
    return nc * 5.0 * math.log2(n ** dim) + 2 * nc * nc + 30.0


def fp64_peak_tflops(reps=3, m=4096):
    """FP64 throughput of this GPU measured in this process: a cuBLAS DGEMM (2 m^3 FLOPs) timed with
    CUDA events, best of `reps` (no setting changed)."""
    import torch
    a = torch.randn(m, m, device="cuda", dtype=torch.float64)
    b = torch.randn(m, m, device="cuda", dtype=torch.float64)
    st = torch.cuda.current_stream()
    torch.matmul(a, b)
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        torch.matmul(a, b)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b
    return 2.0 * m ** 3 / (best / 1e3) / 1e12


def fp32_field_errors(hom, cells, phases, c0):
    """Local-field errors of the FP32 sweep (specialised passes, e_n < 1e-6, the bench's form) against
    the FP64 generic passes converged to e < 1e-10 on the same cells (the FP64 path matches the oracle's
    fields to 1e-10 in the tests): per grid size, the largest over cells, loads and components of the
    relative L2 error (RMS of the difference / RMS of the field) and of the largest error (relative to the
    field's largest magnitude), for eps and sigma."""
    import torch
    mat = hom.hom_filter_build(cells, phases)
    r32 = hom.hom_solve(mat, np.eye(3), c0, precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=TOL,
                        max_iter=MAX_ITER)
    r64 = hom.hom_solve(mat, np.eye(3), c0, precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_E, tol=1e-10,
                        max_iter=MAX_ITER, passes=hom.HOM_PASSES_GENERIC)
    out = {}
    off = 0
    for cell in cells:
        size = 3 * 3 * cell.n ** 2
        per = out.setdefault(str(cell.n), {"eps_l2": 0.0, "eps_max": 0.0, "sigma_l2": 0.0, "sigma_max": 0.0})
        for key in ("eps", "sigma"):
            a = r32[key][off:off + size].double().view(3, 3, -1)
            b = r64[key][off:off + size].view(3, 3, -1)
            d = a - b
            l2 = torch.sqrt((d * d).mean(-1) / (b * b).mean(-1).clamp_min(1e-300)).max().item()
            mx = (d.abs().amax(-1) / b.abs().amax(-1).clamp_min(1e-300)).max().item()
            per[key + "_l2"] = max(per[key + "_l2"], l2)
            per[key + "_max"] = max(per[key + "_max"], mx)
        off += size
    worst = {k: max(v[k] for v in out.values()) for k in ("eps_l2", "eps_max", "sigma_l2", "sigma_max")}
    del r32, r64
    torch.cuda.empty_cache()
    return {"per_n": out, "worst": worst,
            "reference": "FP64 generic passes, e < 1e-10, same cells (matches the oracle's fields to 1e-10 in the tests)"}


def fp64_forms(hom, step, cells, phases, fp32_err):
    """The plain FP64 form of the sweep: one cell at a time (e_n < 1e-6), batched (one call, e_n < 1e-6)
    and batched at the loosest tolerance whose C_eff error against the oracle does not exceed the
    FP32 form's (the metric's "at fixed C_eff error"), with the FP64 ALU fraction of the batched solve."""
    import torch
    gold = golden_ceff()

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, (time.perf_counter() - t) * 1e3

    def vi_of(r, idx):
        return float(sum(cells[i].n ** 2 * it for k, i in enumerate(idx) for it in r["iterations"][k]))

    for i in range(len(cells)):  # warm-up: plans and workspace
        step(precision=hom.HOM_FP64, subset=[i])
    out = {}

    def one_by_one():
        res = [step(precision=hom.HOM_FP64, subset=[i]) for i in range(len(cells))]
        return res
    res, ms = timed(one_by_one)
    vi = sum(vi_of(r, [i]) for i, (r, _) in enumerate(res))
    err, _ = ceff_errors(cells, phases, np.array([r["mean_sigma"][0] for r, _ in res]), gold)
    out["one_cell_at_a_time"] = {"value": vi / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "tol": TOL,
                                 "ceff_max_rel_err": err}
    idx = list(range(len(cells)))
    flops = sum(cells[i].n ** 2 * flops_per_voxel_iteration(cells[i].n) for i in idx)
    for name, tols in (("batched", [TOL]), ("batched_equal_error", [1e-5, 5e-6, 2e-6, TOL])):
        for tol in tols:
            def run(tol=tol):
                import paper_1412_3228_gb300 as h2
                c0 = np.array([H.mean_lame(phases[c.matrix_phase:c.matrix_phase + 2]) for c in cells])
                mat = h2.hom_filter_build(cells, phases)
                return h2.hom_solve(mat, np.eye(3), c0, precision=h2.HOM_FP64, criterion=h2.HOM_CRIT_EN, tol=tol,
                                    max_iter=MAX_ITER, fields=False)
            run()
            r, ms = timed(run)
            vi = vi_of(r, idx)
            err, _ = ceff_errors(cells, phases, r["mean_sigma"], gold)
            fl = float(sum(cells[i].n ** 2 * flops_per_voxel_iteration(cells[i].n) * it
                           for i in idx for it in r["iterations"][i]))
            out[name] = {"value": vi / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "tol": tol, "ceff_max_rel_err": err,
                         "tflops": fl / (ms / 1e3) / 1e12}
            if name == "batched" or (err is not None and fp32_err is not None and err <= fp32_err):
                break
    peak = fp64_peak_tflops()
    for name in ("batched", "batched_equal_error"):
        out[name]["alu"] = {"bound": "alu (fp64)", "peak_tflops": round(peak, 3),
                            "peak_source": "cuBLAS DGEMM 4096^3 timed in this process",
                            "frac": round(out[name]["tflops"] / peak, 4),
                            "flops_model": "per voxel-iteration: 15 log2(n^2) + 48 (FFTs, constitutive, Green)"}
    out["fp32_ceff_max_rel_err"] = fp32_err
    del flops
    return out


def cufft_comparison(hom, cells, phases, c0, dev, reps=10):
    """cuFFT (torch.fft.rfft2 + irfft2) on the real fields of the two 1215^2 cells x 3 loads x 3
    components, and this library's iteration on the same problems (stats of a 4-iteration solve)."""
    import torch
    pick = [i for i, c in enumerate(cells) if c.n == 1215 and c.rule in (H.RULE_VOIGT, H.RULE_TWO_LAYER)
            and abs(phases[c.matrix_phase + 1][1] / phases[c.matrix_phase][1] - 10.0) < 1e-9]
    x = torch.randn(len(pick) * 9, 1215, 1215, device=dev, dtype=torch.float32)
    st = torch.cuda.current_stream()
    for _ in range(3):
        y = torch.fft.irfft2(torch.fft.rfft2(x), s=(1215, 1215))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        y = torch.fft.irfft2(torch.fft.rfft2(x), s=(1215, 1215))
    e1.record(st)
    torch.cuda.synchronize()
    cufft_ms = e0.elapsed_time(e1) / reps
    del x, y
    mat = hom.hom_filter_build([cells[i] for i in pick], phases)
    ms = 0.0
    for _ in range(2):
        r = hom.hom_solve(mat, np.eye(3), c0[pick], precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=-1.0,
                          max_iter=4, fields=False, stats=True)
        ms = sum(r["stats"][k]["ms"] for k in ("row", "green", "control")) / max(1, r["stats"]["green"]["launches"])
    return {"fields": len(pick) * 9, "n": 1215, "cufft_rfft2_irfft2_ms": round(cufft_ms, 4),
            "ours_iteration_ms": round(ms, 4),
            "note": "cuFFT does the forward and inverse transforms only; the iteration also applies the "
                    "constitutive update, Gamma0 and the residual"}


def golden_3d(n):
    p = os.path.join(ROOT, "tests", "golden", "spheres3d_ceff.json")
    if not os.path.exists(p):
        return {}
    return {e["contrast"]: np.array(e["ceff"]) for e in json.load(open(p))["cells"] if e["n"] == n}


def spheres_3d(hom, dev, n=243, contrasts=(10.0,), fp64_check=True):
    """Random-sphere cells of n^3 (volume fraction 0.3, radius U[0.05, 0.1], 2-layer filter r = 1 px,
    8^3 subgrid), one per contrast, 6 Mandel loads each, in one batched FP32 solve to e_n < 1e-6.
    C_eff error: against the oracle's stored values where they exist (tests/golden), else against
    the FP64 generic passes on the same cells to e < 1e-9 (the FP64 path matches the oracle to 1e-8
    at 81^3 and 135^3)."""
    import torch
    base = H.rsa_spheres_cell(n, seed=1000 + n, vf=0.3, rmin=0.05, rmax=0.1, rule=H.RULE_TWO_LAYER,
                              radius_px=1.0, subgrid=8, gap_voxels=n / 243.0)
    phases, cells = [], []
    for contrast in contrasts:
        cells.append(H.remap_phases(base, len(phases)))
        phases.extend(H.two_phases(contrast))
    c0 = np.array([H.mean_lame(phases[2 * i:2 * i + 2]) for i in range(len(cells))])
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    mat = hom.hom_filter_build(cells, phases)  # warm-up
    t0.record(torch.cuda.current_stream())
    mat = hom.hom_filter_build(cells, phases)
    t1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    filt_ms = t0.elapsed_time(t1)
    kw = dict(precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=TOL, max_iter=MAX_ITER, fields=False, stats=True)
    r = hom.hom_solve(mat, np.eye(6), c0, **kw)
    torch.cuda.synchronize()
    t0.record(torch.cuda.current_stream())
    r = hom.hom_solve(mat, np.eye(6), c0, **kw)
    t1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    vi = float(n ** 3 * np.sum(r["iterations"]))
    kb = {k: round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) for k, v in r["stats"].items() if v["ms"] > 0 and v["bytes"] > 0}
    C = hom.hom_effective_stiffness(np.eye(6), r["mean_sigma"], 3)
    gold = golden_3d(n)
    err, ref = None, None
    if all(c in gold for c in contrasts):
        err = max(float(np.abs(C[i] - gold[c]).max() / np.abs(gold[c]).max()) for i, c in enumerate(contrasts))
        ref = "oracle C_eff (tests/golden, e < 1e-9)"
    elif fp64_check:
        r64 = hom.hom_solve(mat, np.eye(6), c0, precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_E, tol=1e-9,
                            max_iter=MAX_ITER, fields=False)
        C64 = hom.hom_effective_stiffness(np.eye(6), r64["mean_sigma"], 3)
        err = max(float(np.abs(C[i] - C64[i]).max() / np.abs(C64[i]).max()) for i in range(len(cells)))
        ref = "FP64 generic passes on the same cells, e < 1e-9"
        del r64
    return {"value": vi / (ms / 1e3), "unit": UNIT, "solve_ms": round(ms, 2), "filter_build_ms": round(filt_ms, 2),
            "cells": len(cells), "contrasts": list(contrasts),
            "iterations": [[int(i) for i in row] for row in r["iterations"]], "spheres": len(base.prims),
            "mixed_voxels": int(mat.mixed_count), "achieved_gbs": kb, "ceff_max_rel_err": err, "ceff_reference": ref,
            "passes": "specialised FP32 3D (row, y forward, Green along z, y inverse)"}


def backward_135(hom, dev, n=135):
    """The differentiation workload: one n^3 random-sphere cell (seed 3000, volume fraction 0.25,
    radius U[0.05, 0.1], contrast 20, 2-layer filter r = 1 px, 8^3 subgrid), FP32 forward solve of the
    6 unit loads (fields kept) and FP32 adjoint solve for L = sum_ij (C_ij - T_ij)^2 / |T|^2 +
    <sigma_vm^2> / <sigma_vm^2>_0 (von Mises term on the xx load; T = C_eff (1 + 0.1 N(0, 1)) symmetrised,
    seed 3001), both on the specialised 3D passes; e_n < 4e-6 (the FP32 floor at contrast 20 is
    near 1.2e-6).  Reports the forward and backward times and the adjoint iterations."""
    import torch
    cell = H.rsa_spheres_cell(n, seed=3000, vf=0.25, rmin=0.05, rmax=0.1, rule=H.RULE_TWO_LAYER, radius_px=1.0,
                              subgrid=8, gap_voxels=n / 243.0)
    phases = H.two_phases(20.0)
    c0 = H.mean_lame(phases)
    st = torch.cuda.current_stream()
    kw = dict(precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=4e-6, max_iter=MAX_ITER)

    def forward():
        mat = hom.hom_filter_build([cell], phases)
        fwd = hom.hom_solve(mat, np.eye(6), c0, **kw)
        return mat, fwd

    def loss_grads(fwd, T=None, vm0=None):
        C = hom.hom_effective_stiffness(np.eye(6), fwd["mean_sigma"], 3)[0]
        s = fwd["sigma"].view(6, 6, -1)[0].double()
        s = s - torch.cat([(s[:3].sum(0, keepdim=True) / 3.0).expand(3, -1), torch.zeros_like(s[3:])])
        vm2 = float(1.5 * (s * s).sum(0).mean())
        if T is None:
            rng = np.random.default_rng(3001)
            T = C * (1.0 + 0.1 * rng.standard_normal(C.shape))
            T = 0.5 * (T + T.T)
            vm0 = vm2
        G = (2.0 * (C - T) / np.sum(T ** 2))[None]
        S = torch.zeros((6, 6, n ** 3), dtype=torch.float32, device="cuda")
        S[0] = (3.0 * s / (n ** 3 * vm0)).float()
        loss = float(np.sum((C - T) ** 2) / np.sum(T ** 2) + vm2 / vm0)
        return G, S, T, vm0, loss

    mat, fwd = forward()  # warm-up, and the target of the loss
    G, S, T, vm0, _ = loss_grads(fwd)
    hom.hom_solve_backward(mat, fwd, c0, dL_dC=G, dL_dsigma=S, want_ctilde=True, want_frac=True, **kw)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(st)
    mat, fwd = forward()
    e[1].record(st)
    G, S, _, _, loss = loss_grads(fwd, T, vm0)
    b = hom.hom_solve_backward(mat, fwd, c0, dL_dC=G, dL_dsigma=S, want_ctilde=True, want_frac=True, **kw)
    e[2].record(st)
    torch.cuda.synchronize()
    return {"n": n, "contrast": 20.0, "loads": 6, "forward_ms": round(e[0].elapsed_time(e[1]), 2),
            "backward_ms": round(e[1].elapsed_time(e[2]), 2), "loss": loss,
            "forward_iterations": [int(i) for i in fwd["iterations"][0]],
            "adjoint_iterations": [int(i) for i in b["adjoint_iterations"][0]],
            "adjoint_status": [int(i) for i in b["adjoint_status"][0]],
            "dL_dphase": b["dphase"].tolist(), "tol": kw["tol"],
            "note": "FP32 forward and adjoint on the specialised 3D passes; loss gradient w.r.t. sigma from torch "
                    "on the returned fields (user side); tests/test_gpu_backward_vm.py checks the gradient "
                    "against finite differences of the FP64 path at this size"}


def cg_comparison(hom, dev, sizes=(135, 405), tol=1e-4):
    """Accelerated schemes against the basic one on the paper's high-contrast cases (section 5): the
    centred disk of radius pi/15 at contrasts 1e3 and 1e-3, n in `sizes`, Voigt and 2-layer filters
    (r = 1 px, S = 16), 3 loads, FP64 (FP32 CG stalls near 1e-2 at contrast 1e3).  The basic scheme
    stops at e_n < tol, conjugate gradients at e_G < tol (e_G >= e_n: at least as strict), the
    Eyre-Milton scheme (reference medium: geometric means of the phase moduli) at max(e_n, e_c) < tol,
    each one batched solve timed with CUDA events after a short warm-up solve; reports the times, the
    iteration counts and the C_eff agreement."""
    import torch
    cells, phases = [], []
    for contrast in (1e3, 1e-3):
        for n in sizes:
            for rule in (H.RULE_VOIGT, H.RULE_TWO_LAYER):
                cell = H.centred_disk_cell(n, rule=rule, radius_px=1.0, subgrid=16, radius=math.pi / 15)
                cells.append(H.remap_phases(cell, len(phases)))
                phases.extend(H.two_phases(contrast))
    c0 = np.array([H.mean_lame(phases[2 * i:2 * i + 2]) for i in range(len(cells))])
    c0_em = np.array([H.geometric_lame(phases[2 * i:2 * i + 2], 2) for i in range(len(cells))])
    mat = hom.hom_filter_build(cells, phases)
    E = np.eye(3)
    st = torch.cuda.current_stream()
    out = {}
    for name in ("fixed_point", "cg", "eyre_milton"):
        def solve(max_iter):
            if name == "cg":
                return hom.hom_solve_cg(mat, E, precision=hom.HOM_FP64, tol=tol, max_iter=max_iter, fields=False)
            if name == "eyre_milton":
                return hom.hom_solve(mat, E, c0_em, precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_EN, tol=tol,
                                     max_iter=max_iter, fields=False, scheme=hom.HOM_SCHEME_EYRE_MILTON)
            return hom.hom_solve(mat, E, c0, precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_EN, tol=tol,
                                 max_iter=max_iter, fields=False)
        solve(20)  # warm-up: plans and workspace
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(st)
        r = solve(4000 if name != "fixed_point" else 30000)
        t1.record(st)
        torch.cuda.synchronize()
        out[name] = dict(ms=round(t0.elapsed_time(t1), 2), iterations_max=int(r["iterations"].max()),
                         iterations_median=float(np.median(r["iterations"])),
                         status_counts={str(k): int(v) for k, v in zip(*np.unique(r["status"], return_counts=True))},
                         C=hom.hom_effective_stiffness(E, r["mean_sigma"], 2))
    Cf, Cc, Ce = out["fixed_point"].pop("C"), out["cg"].pop("C"), out["eyre_milton"].pop("C")
    diff = max(float(np.abs(Cf[i] - Cc[i]).max() / np.abs(Cf[i]).max()) for i in range(len(cells)))
    diff_em = max(float(np.abs(Cf[i] - Ce[i]).max() / np.abs(Cf[i]).max()) for i in range(len(cells)))
    return {"workload": "disk r = pi/15, contrasts 1e3 and 1e-3, n in %s, Voigt and 2-layer, 3 loads, FP64, "
                        "e_n (fixed point) / e_G (CG) < %g" % (list(sizes), tol),
            "cells": len(cells), "fixed_point": out["fixed_point"], "cg": out["cg"], "eyre_milton": out["eyre_milton"],
            "speedup": round(out["fixed_point"]["ms"] / out["cg"]["ms"], 2),
            "speedup_eyre_milton": round(out["fixed_point"]["ms"] / out["eyre_milton"]["ms"], 2),
            "ceff_max_rel_diff": diff, "ceff_max_rel_diff_eyre_milton": diff_em}


def eyre_milton_sweep(hom, cells, phases, c0, fp32_err, reps=3):
    """The sweep's cells by the Eyre-Milton scheme (FP32, specialised passes; reference medium: the
    geometric means of each cell's phase moduli) to max(e_n, e_c) < 1e-6, against the basic scheme
    to e_n < 1e-6, both solves without fields, timed with CUDA events (best of `reps` after a warm-up);
    with each one's C_eff error against the oracle's stored values."""
    import torch
    c0_em = np.array([H.geometric_lame(phases[c.matrix_phase:c.matrix_phase + 2], 2) for c in cells])
    mat = hom.hom_filter_build(cells, phases)
    st = torch.cuda.current_stream()
    kw = dict(precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=TOL, max_iter=MAX_ITER, fields=False)
    out = {}
    for name, c, extra in (("basic", c0, {}), ("eyre_milton", c0_em, {"scheme": hom.HOM_SCHEME_EYRE_MILTON})):
        hom.hom_solve(mat, np.eye(3), c, **kw, **extra)
        best, r = None, None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            r = hom.hom_solve(mat, np.eye(3), c, **kw, **extra)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        err, _ = ceff_errors(cells, phases, r["mean_sigma"], golden_ceff())
        out[name] = {"solve_ms": round(best, 2), "iterations_max": int(r["iterations"].max()),
                     "status_counts": {str(k): int(v) for k, v in zip(*np.unique(r["status"], return_counts=True))},
                     "ceff_max_rel_err_vs_oracle": err}
    out["speedup_time_to_solution"] = round(out["basic"]["solve_ms"] / out["eyre_milton"]["solve_ms"], 2)
    return out


def ensemble_2d(hom, dev, count=256):
    """The batched 2D ensemble: `count` seeded random-disk cells (4-40 disks, volume fraction
    U[0.1, 0.4], grid from {45, 75, 135, 225, 405}, contrast 10^U[-2, 2], Reuss/Voigt/2-layer),
    3 loads each, to e_n < 1e-6, all in one FP32 call.  Beyond contrast ~11 the FP32 iteration's
    rounding floor lies above the tolerance; the production form therefore corrects the pairs that
    stall with FP64 residuals (defect correction, generic passes).  Reported beside it: the plain
    FP32 form on the specialised passes as one graph launch with the autotuned plan and a stagnation
    stop, with the stalled cells finished in FP64 by conjugate gradients.  Both report the time to
    solution of the whole ensemble and their status counts."""
    import torch
    phases, cells = [], []
    for i in range(count):
        cell, ph = H.random_disk_cell(2000 + i)
        cells.append(H.remap_phases(cell, len(phases)))
        phases.extend(ph)
    c0 = np.array([H.mean_lame(phases[2 * i:2 * i + 2]) for i in range(count)])
    st = torch.cuda.current_stream()
    counts = lambda a: {str(k): int(v) for k, v in zip(*np.unique(a, return_counts=True))}
    base = dict(precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=TOL, max_iter=ENSEMBLE_MAX_ITER, fields=False)

    def timed(fn, reps=2):
        for _ in range(reps):  # the first call builds plans, the autotuner's choice and the graph
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            out = fn()
            e1.record(st)
            torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    mat, filt_ms = timed(lambda: hom.hom_filter_build(cells, phases))
    # production form: FP32 with defect correction of the stalled pairs
    r, solve_ms = timed(lambda: hom.hom_solve(mat, np.eye(3), c0, refine=4, **base))
    vi = float(np.sum([[c.n ** 2 * it for it in r["iterations"][i]] for i, c in enumerate(cells)]))
    C = hom.hom_effective_stiffness(np.eye(3), r["mean_sigma"], 2)

    # the other form: specialised passes, graph, autotuner, stagnation stop; FP64 CG for stalled cells
    def stage2(rr):
        redo = [i for i in range(count) if (rr["status"][i] != 0).any()]
        if not redo:
            return None, redo
        sub, sph = [], []
        for i in redo:
            sub.append(H.remap_phases(H.remap_phases(cells[i], -2 * i), len(sph)))
            sph.extend(phases[2 * i:2 * i + 2])
        m2 = hom.hom_filter_build(sub, sph)
        return hom.hom_solve_cg(m2, np.eye(3), precision=hom.HOM_FP64, tol=TOL, max_iter=3000, fields=False), redo
    kw2 = dict(base, use_graph=True, tune=True, stall_window=50)
    r1, fp32_ms = timed(lambda: hom.hom_solve(mat, np.eye(3), c0, **kw2))
    (r2, redo), cg_ms = timed(lambda: stage2(r1))
    final = r1["status"].copy()
    C2 = hom.hom_effective_stiffness(np.eye(3), r1["mean_sigma"], 2)
    if r2 is not None:
        Ccg = hom.hom_effective_stiffness(np.eye(3), r2["mean_sigma"], 2)
        for k, i in enumerate(redo):
            final[i] = r2["status"][k]
            C2[i] = Ccg[k]
    agree = float(max(np.abs(C[i] - C2[i]).max() / np.abs(C2[i]).max() for i in range(count)))
    # the accelerated form: the Eyre-Milton scheme in FP32 (generic passes, one graph launch), the
    # reference medium of each cell the geometric means of its phase moduli
    c0_em = np.array([H.geometric_lame(phases[2 * i:2 * i + 2], 2) for i in range(count)])
    kw3 = dict(base, use_graph=True, stall_window=50, tune=True, scheme=hom.HOM_SCHEME_EYRE_MILTON)
    r3, em_ms = timed(lambda: hom.hom_solve(mat, np.eye(3), c0_em, **kw3))
    C3 = hom.hom_effective_stiffness(np.eye(3), r3["mean_sigma"], 2)
    agree3 = float(max(np.abs(C[i] - C3[i]).max() / np.abs(C[i]).max() for i in range(count)))
    rs = hom.hom_solve(mat, np.eye(3), c0, stall_window=50, stats=True, **base)
    kb = {k: round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) for k, v in rs["stats"].items() if v["ms"] > 0 and v["bytes"] > 0}
    ctr = np.array([max(phases[2 * i + 1][1] / phases[2 * i][1], phases[2 * i][1] / phases[2 * i + 1][1])
                    for i in range(count)])
    return {"value": vi / (solve_ms / 1e3), "unit": UNIT, "solve_ms": round(solve_ms, 2),
            "filter_build_ms": round(filt_ms, 2), "time_to_solution_ms": round(filt_ms + solve_ms, 2),
            "cells": count, "voxels": int(sum(c.n ** 2 for c in cells)), "phases": len(phases),
            "iterations": {"max": int(r["iterations"].max()), "median": float(np.median(r["iterations"])),
                           "min": int(r["iterations"].min())},
            "status_counts": counts(r["status"]), "err_n_max": float(r["err_n"].max()),
            "form": "FP32, one call; pairs stalled at the FP32 floor corrected with FP64 residuals (refine = 4, generic passes)",
            "fp32_then_fp64_cg": {"fp32_solve_ms": round(fp32_ms, 2), "fp64_cg_ms": round(cg_ms, 2),
                                  "time_to_solution_ms": round(filt_ms + fp32_ms + cg_ms, 2),
                                  "fp32_status_counts": counts(r1["status"]), "cells_finished_in_fp64_cg": len(redo),
                                  "final_status_counts": counts(final),
                                  "form": "specialised passes, one graph launch, autotuned plan, stagnation stop 50; "
                                          "stalled cells by FP64 conjugate gradients"},
            "eyre_milton_fp32": {"solve_ms": round(em_ms, 2), "time_to_solution_ms": round(filt_ms + em_ms, 2),
                                 "status_counts": counts(r3["status"]),
                                 "iterations": {"max": int(r3["iterations"].max()),
                                                "median": float(np.median(r3["iterations"]))},
                                 "err_n_max": float(r3["err_n"].max()), "err_c_max": float(r3["err_c"].max()),
                                 "ceff_max_rel_diff_to_production_form": agree3,
                                 "form": "Eyre-Milton scheme (c0: geometric means of the phase moduli), FP32, one graph "
                                         "launch, autotuned plan; stops at max(e_n, e_c) < tol"},
            "ceff_max_rel_diff_between_forms": agree,
            "stalled_cells_min_contrast": float(ctr[redo].min()) if redo else None,
            "achieved_gbs_fp32_specialised": kb}


def cpu_model():
    """The host CPU's model name (x86 /proc/cpuinfo, else lscpu, e.g. on Arm hosts)."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_job(job):
    """One oracle run (in a spawned worker or the main process); returns its voxel-iterations and time.
    ("solve2d", n, contrast, rule, loads, tol, criterion): filter build + full solve of the centred
    disk (volume fraction 0.2, r = 1 px, 16x16 subgrid) for the first `loads` unit Mandel loads;
    ("iter3d", n, iters): `iters` fixed iterations of one load on an n^3 laminate (no filter)."""
    import oracle as O
    t = time.perf_counter()
    if job[0] == "solve2d":
        _, n, contrast, rule, loads, tol, crit = job
        phases = H.two_phases(contrast)
        cell = H.centred_disk_cell(n, vf=0.2, rule=rule, radius_px=1.0, subgrid=16)
        fb = O.filter_build(cell, phases)
        lam0, mu0 = H.mean_lame(phases)
        r = O.solve(fb["ctilde"], 2, n, lam0, mu0, np.eye(3)[:loads], tol=tol, max_iter=MAX_ITER, criterion=crit)
        its = [int(i) for i in r["iterations"]]
        return {"job": list(job), "vi": float(n * n * sum(its)), "iterations": its, "seconds": time.perf_counter() - t}
    _, n, iters = job
    phases = H.two_phases(10.0)
    fb = O.filter_build(H.laminate_cell(n, 3, 0.3), phases)
    lam0, mu0 = H.mean_lame(phases)
    t = time.perf_counter()
    O.solve(fb["ctilde"], 3, n, lam0, mu0, np.eye(6)[:1], tol=-1.0, max_iter=iters)
    return {"job": list(job), "vi": float(n ** 3 * iters), "seconds": time.perf_counter() - t}


def cpu_baseline(args, pool=None):
    """The FP64 oracle as it stands on this machine's host cores, on bounded samples of the workloads:
    single core -- full solves of the 45^2 cell of the first configuration (one load, e < 1e-8), of
    the sweep's eight 45^2 cells and of two of its 135^2 cells (3 loads, e_n < 1e-6);
    all cores -- the sweep's eight 405^2 cells solved in parallel (one worker per cell, `pool`);
    3D -- one fixed iteration of one load on a 135^3 cell (time per iteration).
    The 1215^2 cells and full 3D solves take hours on a host core and are left out."""
    import oracle as O
    jobs1 = [("solve2d", 45, 10.0, H.RULE_VOIGT, 1, 1e-8, O.CRIT_E)]
    jobs1 += [("solve2d", 45, c, r, 3, TOL, O.CRIT_EN) for c in CONTRASTS for r in RULES]
    jobs1 += [("solve2d", 135, 10.0, H.RULE_VOIGT, 3, TOL, O.CRIT_EN), ("solve2d", 135, 0.1, H.RULE_REUSS, 3, TOL, O.CRIT_EN)]
    all_core = third = None
    pending = None
    if pool is not None:
        jobs_all = [("solve2d", 405, c, r, 3, TOL, O.CRIT_EN) for c in CONTRASTS for r in RULES]
        t_all = time.perf_counter()
        pending = pool.map_async(oracle_job, jobs_all)
        pending3 = pool.apply_async(oracle_job, (("iter3d", 135, 1),))
    t = time.perf_counter()
    res1 = [oracle_job(j) for j in jobs1]
    dt1 = time.perf_counter() - t
    vi1 = sum(r["vi"] for r in res1)
    per_filter = {}
    for r in res1[1:]:
        per_filter.setdefault(H.RULE_NAMES[r["job"][3]], []).extend(r["iterations"])
    if pending is not None:
        ra = pending.get()
        dt_all = time.perf_counter() - t_all
        for r in ra:
            per_filter.setdefault(H.RULE_NAMES[r["job"][3]], []).extend(r["iterations"])
        all_core = {"value": sum(r["vi"] for r in ra) / dt_all, "unit": UNIT, "cores": min(len(jobs_all), os.cpu_count() or 1),
                    "sample": "the sweep's eight 405^2 cells (3 loads, e_n < %g), one worker per cell, %.1f s" % (TOL, dt_all)}
        r3 = pending3.get()
        third = {"n": 135, "seconds_per_iteration": r3["seconds"], "value": r3["vi"] / r3["seconds"], "unit": UNIT,
                 "sample": "1 fixed iteration, one load, 135^3 laminate (iteration cost does not depend on geometry)"}
    return {"value": vi1 / dt1, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "full solves: 45^2 disk (1 load, e < 1e-8), the sweep's eight 45^2 cells and its 135^2 Voigt "
                      "(contrast 10) and Reuss (0.1) cells (3 loads, e_n < %g), filter build included, %.1f s on one "
                      "core" % (TOL, dt1),
            "cpu_model": cpu_model(), "nproc": os.cpu_count(), "all_cores": all_core, "per_iteration_3d": third,
            "iterations_per_filter": {k: {"median": float(np.median(v)), "max": int(max(v))} for k, v in per_filter.items()}}


def reference_sample():
    """One bounded step of the reference arm: the oracle's filter build and 2 fixed iterations of the
    3 loads of the sweep's 405^2 Voigt cell (contrast 10), on one host core."""
    import oracle as O
    cells, phases, c0 = workload()
    idx = [i for i, c in enumerate(cells) if c.n == 405 and c.rule == H.RULE_VOIGT][0]
    cell = cells[idx]
    t = time.perf_counter()
    fb = O.filter_build(cell, phases)
    O.solve(fb["ctilde"], 2, cell.n, c0[idx][0], c0[idx][1], np.eye(3), tol=-1.0, max_iter=2)
    return cell.n ** 2 * 2 * 3 / (time.perf_counter() - t)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on a bounded sample of the workload per step."""
    for _ in range(args.warmup):
        reference_sample()
    t = time.perf_counter()
    vals = [reference_sample() for _ in range(args.steps)]
    dt = time.perf_counter() - t
    value = float(np.mean(vals))
    sample = "405^2 Voigt cell of the sweep, contrast 10: oracle filter build + 3 loads x 2 iterations per step"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict({"sample": sample}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def profile_case(args):
    """Small fixed case for ncu captures: two 1215^2 cells (Voigt and 2-layer, contrast 10), 3 loads,
    exactly `args.iters` fixed-point iterations in FP32 (or FP64 with --fp64-case)."""
    import torch

    import paper_1412_3228_gb300 as hom
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)
    cells, phases, c0 = workload()
    pick = [i for i, c in enumerate(cells) if c.n == args.profile_n and c.rule in (H.RULE_VOIGT, H.RULE_TWO_LAYER)
            and abs(phases[c.matrix_phase + 1][1] / phases[c.matrix_phase][1] - 10.0) < 1e-9]
    mat = hom.hom_filter_build([cells[i] for i in pick], phases)
    prec = hom.HOM_FP64 if args.fp64_case else hom.HOM_FP32
    r = hom.hom_solve(mat, np.eye(3), c0[pick], precision=prec, criterion=hom.HOM_CRIT_EN, tol=-1.0,
                      max_iter=args.iters, fields=False)
    torch.cuda.synchronize()
    print("profile case: %d cells of n=%d, %d iterations, status %s" % (len(pick), args.profile_n, args.iters,
                                                                          r["status"].ravel().tolist()))


def profile_case3d(args):
    """Small fixed 3D case for ncu captures: one 135^3 random-sphere cell (2-layer filter, contrast
    10), 6 loads, exactly `args.iters` fixed-point iterations in FP32 (state ~380 MB per buffer)."""
    import torch

    import paper_1412_3228_gb300 as hom
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)
    n = 135
    cell = H.rsa_spheres_cell(n, seed=1000 + n, vf=0.3, rmin=0.05, rmax=0.1, rule=H.RULE_TWO_LAYER,
                              radius_px=1.0, subgrid=8, gap_voxels=n / 243.0)
    phases = H.two_phases(10.0)
    mat = hom.hom_filter_build([cell], phases)
    r = hom.hom_solve(mat, np.eye(6), np.array([H.mean_lame(phases)]), precision=hom.HOM_FP32,
                      criterion=hom.HOM_CRIT_EN, tol=-1.0, max_iter=args.iters, fields=False)
    torch.cuda.synchronize()
    print("profile case 3d: one cell of n=%d, %d iterations, status %s" % (n, args.iters, r["status"].ravel().tolist()))


def profile_cg(args):
    """Small fixed case for ncu captures of the conjugate-gradient path: one n^2 Voigt disk
    (n = --profile-n, radius pi/15, contrast 1e3), 3 loads, FP64, exactly `args.iters` CG steps
    (n = 1215: each mixed-domain field is 106 MB, above L2; about 0.7 GB on the device)."""
    import torch

    import paper_1412_3228_gb300 as hom
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)
    cell = H.centred_disk_cell(args.profile_n, rule=H.RULE_VOIGT, radius=math.pi / 15)
    mat = hom.hom_filter_build([cell], H.two_phases(1e3))
    r = hom.hom_solve_cg(mat, np.eye(3), precision=hom.HOM_FP64, tol=1e-30, max_iter=args.iters, fields=False)
    torch.cuda.synchronize()
    print("profile cg: one %d^2 cell, %d CG steps, status %s" % (args.profile_n, args.iters, r["status"].ravel().tolist()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-case", action="store_true", help="run only the small fixed ncu case")
    ap.add_argument("--profile-case3d", action="store_true", help="run only the small fixed 3D ncu case")
    ap.add_argument("--profile-cg", action="store_true", help="run only the small fixed conjugate-gradient ncu case")
    ap.add_argument("--profile-n", type=int, default=1215)
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--fp64-case", action="store_true")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-cufft", action="store_true")
    ap.add_argument("--skip-3d", action="store_true")
    ap.add_argument("--skip-ensemble", action="store_true")
    ap.add_argument("--skip-cg", action="store_true")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.profile_case:
        profile_case(args)
        return
    if args.profile_cg:
        profile_cg(args)
        return
    if args.profile_case3d:
        profile_case3d(args)
        return
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
