#!/usr/bin/env python
"""Benchmark of the even-odd Wilson-clover solve on one GB300 (or N replicas).

Workload (synthetic, seeded): 32^3 x 64 lattice, links exp(i 0.4 H) (gauge
seed 3), kappa 0.1355, csw 1.0 (four-leaf clover), Gaussian source (seed 0),
antiperiodic t; mixed-precision even-odd CG on the normal equations: FP16
spinor storage with per-site norms, FP32 links (recon-12) and clover, FP32
arithmetic inside, FP64 reliable update whenever the iterated residual has
fallen by 10 since the last one (and at least every 100 iterations), stopped
at true residual |b - M x|/|b| <= 1e-10.  (With the links and clover in FP16 too the
operator's rounding, amplified by the condition number of the normal
equations, triples the iteration count; that variant is timed as well.)

One step = one complete solve (b and the solution resident in HBM; the
gauge field and the clover term are set up beforehand).  The metric is the
sustained dslash rate of the solve: hopping applications x 1320 flops x V/2
sites / wall time.  Also reported: the dslash kernels' achieved HBM
bandwidth against the measured copy bandwidth (roofline), the end-to-end
rate through lqcd_solve with host buffers, solve times of the plain FP64
CG and of every other inner storage on the same system, a stand-alone FP32
recon-12 dslash rate, and the FP64 CPU oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (the solve does not
shard across GPUs here): weak scaling, no collective on the data path.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Dslash GFLOP/s & % HBM roofline; solve time to 1e-10 resid vs plain FP64 CG"
WORKLOADS = {
    "32c64": dict(dims=(32, 32, 32, 64), eps=0.4, gauge_seed=3, src_seed=0, kappa=0.1355, csw=1.0),
    "16c32": dict(dims=(16, 16, 16, 32), eps=0.5, gauge_seed=2, src_seed=0, kappa=0.135, csw=1.0),
    # larger than L2, a few GB on the device: the size used for kernel captures
    "24c48": dict(dims=(24, 24, 24, 48), eps=0.4, gauge_seed=3, src_seed=0, kappa=0.1355, csw=1.0),
}
TOL = 1e-10
# FP64 residual replacement: every RELIABLE_EVERY iterations or when |r| has
# fallen below RELIABLE_DELTA times its largest value since the last one
# (measured at 32^3x64, FP16 spinors: 100 / 0.1 took 380 iterations and 7
# replacements in 290 ms; 50 / 0.1 took 390 and 9 in 306 ms)
RELIABLE_EVERY, RELIABLE_DELTA = 100, 0.1
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes (read + write) per output site of the inner hopping kernels,
# from one ncu capture of a CG iteration on 24^3x48 (the four launches of an
# iteration: Mhat sweeps with A^-1 and x-pay + norm epilogues, Mhat^dag sweeps
# with A^-1 and the fused CG update); traffic grows with the sites processed.
DRAM_BYTES_PER_SITE = {"f16spinors": (765.3 + 820.3 + 765.6 + 1151.4) / 4}
STORAGE = {
    "f32": "f32 spinors, links (recon-12) and clover",
    "f16": "f16 spinors (per-site norm), links (recon-12) and clover",
    "bf16": "bf16 spinors (per-site norm), links (recon-12) and clover",
    "f16links": "f16 links (recon-12) and clover, f32 spinors",
    "bf16links": "bf16 links (recon-12) and clover, f32 spinors",
    "f16spinors": "f16 spinors (per-site norm), f32 links (recon-12) and clover",
    "bf16spinors": "bf16 spinors (per-site norm), f32 links (recon-12) and clover",
}


def workload_name(w):
    d = w["dims"]
    return ("wilson-clover even-odd CG-NE %dx%dx%dx%d, exp(i %.1f H) links, kappa %.4g, csw %.1f, "
            "tol 1e-10" % (d[0], d[1], d[2], d[3], w["eps"], w["kappa"], w["csw"]))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------- replica aggregation
# Each rank solves its own copy of the workload (the solve does not shard
# across GPUs here); the job's time is the slowest rank's, its work the sum.

def reduce_max(value, device):
    import torch
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value, device):
    import torch
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ our arm

def run_ours(args, w, rank, world, local_rank):
    import torch

    import synth
    from paper_1103_1363_gb300 import lqcd

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dims = w["dims"]
    V = int(np.prod(dims))
    Vh = V // 2
    U = synth.smooth_gauge(dims, w["eps"], w["gauge_seed"])
    b = synth.gaussian_spinor(dims, w["src_seed"])
    stream = torch.cuda.Stream(device=dev)
    lat = lqcd.Lattice(dims, precisions=("f64", "f32", "f16", "bf16", "f16links", "bf16links"), recon=12,
                       device=dev,
                       stream=stream)
    with torch.cuda.stream(stream):
        Ud = torch.from_numpy(U).to(dev)
        bd = torch.from_numpy(b).to(dev)
        xd = torch.zeros_like(bd)
    stream.synchronize()
    lat.gauge_load(Ud)
    t0 = time.time()
    lat.clover_compute(w["kappa"], w["csw"])
    clover_s = time.time() - t0
    # block sizes (plain, plain reducing, dagger, dagger reducing)
    tuned = {p: lqcd.lqcd_tune(lat.ctx, p) for p in ("f64", args.inner)}
    del Ud
    params = dict(inner_prec=args.inner, reliable_interval=RELIABLE_EVERY, reliable_delta=RELIABLE_DELTA,
                  check_interval=10)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        lat.solve(xd, bd, TOL, **params)
    lqcd.lqcd_profile_enable(lat.ctx, True)
    lqcd.lqcd_profile_read(lat.ctx)
    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    stream.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = []
    for _ in range(args.steps):
        _, st = lat.solve(xd, bd, TOL, **params)
        stats.append(st)
    ev1.record(stream)
    stream.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = lqcd.lqcd_profile_read(lat.ctx)
    lqcd.lqcd_profile_enable(lat.ctx, False)
    ms = reduce_max(ms, dev)
    dslash_total = sum(s["dslash_count"] for s in stats)
    flops = reduce_sum(dslash_total * 1320.0 * Vh, dev)
    value = flops / (ms * 1e-3) / 1e9
    worst_res = max(s["true_residual"] for s in stats)
    launches = sum(s["kernel_launches"] for s in stats)

    # dominant kernel: the hopping kernels of the inner precision (all epilogues) inside the solve
    hb, hbsrc = measured_peaks()
    pf = prof[args.inner]
    achieved = pf["bytes"] / (pf["ms"] * 1e-3) / 1e9 if pf["ms"] > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": "dslash_kernel (%s storage, recon-12; all epilogues of the solve)"
                % args.inner,
                "achieved": round(achieved, 1), "peak": hb, "unit": "GB/s",
                "frac": round(achieved / hb, 4), "peak_source": hbsrc,
                "launches": pf["launches"], "avg_launch_us": round(1e3 * pf["ms"] / max(1, pf["launches"]), 2),
                "kernel_time_share": round(sum(p["ms"] for p in prof.values()) / (ms / world if world > 1 else ms), 4),
                "traffic": None}
    if args.inner in DRAM_BYTES_PER_SITE:
        roofline["traffic"] = round(DRAM_BYTES_PER_SITE[args.inner] * Vh)
        roofline["traffic_note"] = ("bytes per launch: ncu dram read+write per output site on 24^3x48, mean over the "
                                    "four launches of an iteration, times V/2; algorithmic bytes per launch here %d"
                                    % round(pf["bytes"] / max(1, pf["launches"])))

    out = {"value": value, "ms": ms, "stats": stats, "roofline": roofline, "clocks": clk,
           "dslash_total": dslash_total, "worst_res": worst_res, "launches": launches,
           "clover_setup_s": round(clover_s, 3), "prof": prof, "tuned": tuned}

    if rank == 0 and not args.quick:
        out["e2e"] = guarded("e2e", e2e_leg, args, lat, b, Vh, params)
        out["solve"] = guarded("solve", compare_solves, lat, bd, xd, stream, params)
        out["dslash_f32"] = guarded("dslash_f32", dslash_microbench, lat, b, dims, stream, hb, hbsrc)
        out["alu_peaks"] = guarded("alu_peaks", alu_peaks, local_rank)
    lat.close()
    if rank == 0 and not args.quick:
        del bd, xd
        torch.cuda.empty_cache()
        out["multi_rhs"] = guarded("multi_rhs", multi_rhs_leg, dev)
        if not args.skip_learned:
            out["learned"] = guarded("learned", learned_leg, dev)
    return out


def guarded(name, fn, *args):
    """A comparison leg: its failure is reported in its place (and on
    stderr) instead of costing the run its JSON line."""
    try:
        return fn(*args)
    except Exception as ex:  # noqa: BLE001 - any failure of a side measurement
        msg = "%s: %s" % (type(ex).__name__, ex)
        print("bench: leg %s failed: %s" % (name, msg), file=sys.stderr, flush=True)
        return {"error": msg[:300]}


def e2e_leg(args, lat, b, Vh, params):
    """Same metric through lqcd_solve with pinned host b and x: the H2D copy
    of b and the D2H copy of x are inside each timed step."""
    import torch
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    lat.solve(xh, bh, TOL, **params)
    t0 = time.perf_counter()
    total = 0
    for _ in range(args.steps):
        _, st = lat.solve(xh, bh, TOL, **params)
        total += st["dslash_count"]
    dt = time.perf_counter() - t0
    nbytes = bh.numel() * bh.element_size()
    return {"value": total * 1320.0 * Vh / dt / 1e9, "unit": "GFLOP/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "ms_per_step": round(1e3 * dt / args.steps, 3)}


def compare_solves(lat, bd, xd, stream, params):
    """One solve per inner precision (outside the timed region), each timed
    with CUDA events on the context stream."""
    import torch
    res = {}
    for name, kw in (("f16_inner_f64_ru", dict(params, inner_prec="f16")),
                     ("bf16_inner_f64_ru", dict(params, inner_prec="bf16")),
                     ("f16links_inner_f64_ru", dict(params, inner_prec="f16links")),
                     ("bf16links_inner_f64_ru", dict(params, inner_prec="bf16links")),
                     ("f16spinors_inner_f64_ru", dict(params, inner_prec="f16spinors")),
                     ("bf16spinors_inner_f64_ru", dict(params, inner_prec="bf16spinors")),
                     ("f32_inner_f64_ru", dict(params, inner_prec="f32")),
                     ("plain_f64_cg", dict(inner_prec="f64", check_interval=10))):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        rc, st = lat.solve(xd, bd, TOL, raise_on_error=False, **kw)
        e1.record(stream)
        stream.synchronize()
        res[name] = {"seconds": round(e0.elapsed_time(e1) * 1e-3, 4), "iterations": st["iterations"],
                     "reliable_updates": st["reliable_updates"], "dslash": st["dslash_count"],
                     "true_residual": st["true_residual"], "status": rc,
                     "precision_fallback": st["precision_fallback"]}
    f64 = res["plain_f64_cg"]["seconds"]
    for k in res:
        res[k]["speedup_vs_f64_cg"] = round(f64 / res[k]["seconds"], 2)
    return res


def timed_solves(lat, stream, calls):
    """Run calls() (a list of (x, b, kw) solves) once for warm-up and once
    timed with CUDA events on the context stream; returns seconds and the
    stats of the timed solves."""
    import torch
    for x, bb, kw in calls:
        lat.solve(x, bb, TOL, raise_on_error=False, **kw)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sts = []
    for x, bb, kw in calls:
        rc, st = lat.solve(x, bb, TOL, raise_on_error=False, **kw)
        st["status"] = rc
        sts.append(st)
    e1.record(stream)
    stream.synchronize()
    return e0.elapsed_time(e1) * 1e-3, sts


def multi_rhs_leg(dev):
    """The 12 point sources (every spin and colour at the origin) on 24^3x48,
    links exp(i 0.5 H) (seed 4), kappa 0.135, csw 1: one multi-right-hand-side
    solve (FP16 spinors, FP32 links and FP32 inner, FP64 reliable updates,
    graph replay) against 12 single-source solves of the same kind and 12
    plain FP64 GPU CG solves; every solve to true residual 1e-10.  Then the
    uneven batch 8^4 (kappa 0.12) + 12^4 (0.1275) + 16^3x32 (0.135) in one
    graph-captured lqcd_solve_batch against the three solved one after the
    other."""
    import torch

    import synth
    from paper_1103_1363_gb300 import lqcd
    dims = (24, 24, 24, 48)
    kappa, csw = 0.135, 1.0
    stream = torch.cuda.Stream(device=dev)
    lat = lqcd.Lattice(dims, precisions=("f64", "f32"), max_nrhs=12, device=dev, stream=stream)
    lat.gauge_load(torch.from_numpy(synth.smooth_gauge(dims, 0.5, 4)).to(dev))
    lat.clover_compute(kappa, csw)
    srcs = np.stack([synth.point_source(dims, s, c) for s in range(4) for c in range(3)])
    b = torch.from_numpy(srcs).to(dev)
    x = torch.zeros_like(b)
    res = {"workload": "12 point sources, 24x24x24x48, exp(i 0.5 H) links, kappa 0.135, csw 1.0, tol 1e-10"}
    mixed = dict(reliable_interval=RELIABLE_EVERY, reliable_delta=RELIABLE_DELTA, check_interval=10, use_graph=1)

    def summary(t, sts):
        return {"seconds": round(t, 4), "iterations_max": max(s["iterations"] for s in sts),
                "true_residual_max": max(s["true_residual"] for s in sts),
                "all_converged": all(s["status"] == 0 for s in sts),
                "launches": sum(s["kernel_launches"] for s in sts)}

    for name, kw in (("multi_rhs_f16spinors", dict(mixed, inner_prec="f16spinors")),
                     ("multi_rhs_f16spinors_persistent", dict(mixed, inner_prec="f16spinors", persistent=1)),
                     ("multi_rhs_f32", dict(mixed, inner_prec="f32"))):
        t, sts = timed_solves(lat, stream, [(x, b, dict(kw, nrhs=12))])
        res[name] = summary(t, sts)
    for name, kw in (("single_rhs_f16spinors_x12", dict(mixed, inner_prec="f16spinors")),
                     ("plain_f64_cg_x12", dict(inner_prec="f64", check_interval=10))):
        t, sts = timed_solves(lat, stream, [(x[r], b[r], kw) for r in range(12)])
        res[name] = summary(t, sts)
    f64 = res["plain_f64_cg_x12"]["seconds"]
    for k in list(res):
        if isinstance(res[k], dict):
            res[k]["speedup_vs_f64_cg"] = round(f64 / res[k]["seconds"], 2)
    lat.close()
    del x, b

    specs = [((8, 8, 8, 8), 0.120, 4), ((12, 12, 12, 12), 0.1275, 5), ((16, 16, 16, 32), 0.135, 6)]
    lats, xs, bs = [], [], []
    for d, kap, seed in specs:
        l = lqcd.Lattice(d, precisions=("f64", "f32"), device=dev, stream=stream)
        l.gauge_load(torch.from_numpy(synth.smooth_gauge(d, 0.5, seed)).to(dev))
        l.clover_compute(kap, 1.0)
        lats.append(l)
        bs.append(torch.from_numpy(synth.gaussian_spinor(d, seed + 100)).to(dev))
        xs.append(torch.zeros_like(bs[-1]))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ub = {"lattices": ["%dx%dx%dx%d kappa %.4g" % (d + (k,)) for d, k, _ in specs], "inner": "f32"}
    for name, p in (("batch_one_graph", lqcd.solver_params(inner_prec="f32", use_graph=1)),
                    ("batch_persistent", lqcd.solver_params(inner_prec="f32", persistent=1))):
        for rep in range(2):  # warm-up, timed
            stream.synchronize()
            e0.record(stream)
            rc, st = lqcd.lqcd_solve_batch([l.ctx for l in lats], xs, bs, [TOL] * 3, p, raise_on_error=False)
            e1.record(stream)
            stream.synchronize()
        ub[name] = {"seconds": round(e0.elapsed_time(e1) * 1e-3, 4), "status": rc,
                    "iterations": [s["iterations"] for s in st],
                    "true_residual": [s["true_residual"] for s in st],
                    "launches": sum(s["kernel_launches"] for s in st)}
    seq = []
    for rep in range(2):
        stream.synchronize()
        e0.record(stream)
        seq = [l.solve(xx, bb, TOL, raise_on_error=False, inner_prec="f32", use_graph=1)[1]
               for l, xx, bb in zip(lats, xs, bs)]
        e1.record(stream)
        stream.synchronize()
    ub["one_after_the_other"] = {"seconds": round(e0.elapsed_time(e1) * 1e-3, 4),
                                 "iterations": [s["iterations"] for s in seq],
                                 "seconds_each": [round(s["seconds"], 4) for s in seq],
                                 "true_residual": [s["true_residual"] for s in seq],
                                 "launches": sum(s["kernel_launches"] for s in seq)}
    for l in lats:
        l.close()
    res["uneven_batch"] = ub
    return res


def learned_leg(dev):
    """The learned-preconditioner workload (16^4, links exp(i 0.5 H), kappa
    0.134, csw 1): pairs from 24 training fields (4096, 20-iteration CG),
    training of the 1-12-12-1 BF16 network (10 epochs, batch 16, Adam lr
    1e-3), then on 8 held-out fields FGCR(20) with the trained network, the
    untrained one, the identity and SAP against even-odd CG (FP32 and
    FP16-spinor inner), each to true residual 1e-10."""
    from paper_1103_1363_gb300 import learned
    out = learned.run_experiment(device=dev, log=lambda *a: None)
    return {"workload": "16^4, 24 training + 8 held-out fields, exp(i 0.5 H), kappa 0.134, csw 1.0, "
                        "net 1-12-12-1 BF16, FGCR(20), tol 1e-10",
            "pairs_s": round(out["pairs_s"], 2), "train_s": round(out["train_s"], 2),
            "loss_first_last": [out["loss_history"][0], out["loss_history"][-1]],
            "solvers": {k: {"iterations_mean": v["iterations_mean"], "ms_mean": round(1e3 * v["wall_s_mean"], 2),
                            "true_residual_max": v["true_residual_max"], "all_converged": v["all_converged"]}
                        for k, v in out["summary"].items()}}


def dslash_microbench(lat, b, dims, stream, hb, hbsrc):
    """FP32 recon-12 parity hopping term alone: 8 buffer pairs rotated
    (8 x 302 MB > L2), 50 timed launches after 5 warm-ups."""
    import torch
    Vh = int(np.prod(dims)) // 2
    nbuf = 8
    with torch.cuda.stream(stream):
        fins = [lat.new_field("f32") for _ in range(nbuf)]
        fouts = [lat.new_field("f32") for _ in range(nbuf)]
    for f in fins:
        lat.pack(f, b, 1, "f32")
    for i in range(5):
        lat.dslash(fouts[i % nbuf], fins[i % nbuf], 0, prec="f32")
    stream.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n = 50
    e0.record(stream)
    for i in range(n):
        lat.dslash(fouts[i % nbuf], fins[i % nbuf], 0, prec="f32")
    e1.record(stream)
    stream.synchronize()
    t = e0.elapsed_time(e1) * 1e-3 / n
    comp = 576.0 * Vh  # FP32 recon-12 compulsory bytes per launch
    return {"gflops": round(1320.0 * Vh / t / 1e9, 1), "us_per_launch": round(t * 1e6, 2),
            "compulsory_bytes": comp, "achieved_gbs": round(comp / t / 1e9, 1),
            "time_roofline_frac": round(comp / t / 1e9 / hb, 4), "peak": hb, "peak_source": hbsrc}


def alu_peaks(device):
    """The device's measured multiply-add peaks (lqcd_fma_peak), TFLOP/s: the
    denominators of the kernels bound by FP32 or FP64 arithmetic."""
    from paper_1103_1363_gb300 import lqcd
    return {"fp32_fma_tflops": round(lqcd.lqcd_fma_peak(device, 0), 1),
            "fp32x2_fma_tflops": round(lqcd.lqcd_fma_peak(device, 1), 1),
            "fp64_fma_tflops": round(lqcd.lqcd_fma_peak(device, 2), 3),
            "source": "measured by lqcd_fma_peak: independent multiply-add chains, 2048 threads per SM"}


def run_hop_kernel(args, w):
    """Stand-alone parity hopping term (recon-12) of one precision, for kernel
    profiles: warmup + steps launches over rotating buffer pairs, each holding
    --nrhs right-hand sides (one launch serves all of them; the compulsory
    bytes count the links once per launch)."""
    import torch

    import synth
    from paper_1103_1363_gb300 import lqcd
    dims = w["dims"]
    Vh = int(np.prod(dims)) // 2
    R = args.nrhs  # the hopping term takes any nrhs; the context's solver vectors are not used
    stream = torch.cuda.Stream()
    U = torch.from_numpy(synth.smooth_gauge(dims, w["eps"], w["gauge_seed"])).cuda()
    b = synth.gaussian_spinor(dims, w["src_seed"])
    nbuf = 8 if R == 1 else 3
    spinor = {"f64": 192, "f32": 96, "f16": 52, "bf16": 52, "f16links": 96, "bf16links": 96, "f16spinors": 52,
              "bf16spinors": 52}
    link = {"f64": 144, "f32": 48, "f16": 24, "bf16": 24, "f16links": 24, "bf16links": 24, "f16spinors": 48,
            "bf16spinors": 48}
    hb, src = measured_peaks()
    lat = lqcd.Lattice(dims, precisions=("f64", "f32", args.prec), recon=args.recon, stream=stream)
    lat.gauge_load(U)
    if args.staged:  # the shared-memory staged kernel for the plain launches
        lqcd.lqcd_tune_set(lat.ctx, args.prec, (lqcd.BLOCK_STAGED, 128, lqcd.BLOCK_STAGED, 128))
    with torch.cuda.stream(stream):
        fins = [lat.new_field(args.prec, nrhs=R) for _ in range(nbuf)]
        fouts = [lat.new_field(args.prec, nrhs=R) for _ in range(nbuf)]
    bb = np.broadcast_to(b, (R,) + b.shape).copy()
    for f in fins:
        lat.pack(f, bb, 1, args.prec, nrhs=R)
    for i in range(args.warmup):
        lat.dslash(fouts[i % nbuf], fins[i % nbuf], 0, prec=args.prec, nrhs=R)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        lat.dslash(fouts[i % nbuf], fins[i % nbuf], 0, prec=args.prec, nrhs=R)
    e1.record(stream)
    stream.synchronize()
    t = e0.elapsed_time(e1) * 1e-3 / args.steps
    sb = spinor[args.prec]
    lb = link[args.prec] * (args.recon / 12.0 if args.prec != "f64" else 1)
    comp = (2 * sb * R + 8 * lb) * Vh
    extra = {}
    if args.prec == "f64":  # FP64-pipe-bound: the arithmetic roofline as well
        pk = lqcd.lqcd_fma_peak(torch.cuda.current_device(), 2)
        extra = {"alu_tflops": round(1320.0 * Vh * R / t / 1e12, 3), "fp64_peak_tflops": round(pk, 3),
                 "alu_frac": round(1320.0 * Vh * R / t / 1e12 / pk, 4)}
    print(json.dumps({"kernel": "hop", "variant": "staged" if args.staged else "gather", "prec": args.prec,
                      "recon": args.recon, "nrhs": R, **extra,
                      "workload": workload_name(w),
                      "us_per_launch": round(t * 1e6, 2), "us_per_rhs": round(t * 1e6 / R, 2),
                      "gflops": round(1320.0 * Vh * R / t / 1e9, 1),
                      "compulsory_bytes": comp, "achieved_gbs": round(comp / t / 1e9, 1),
                      "frac": round(comp / t / 1e9 / hb, 4), "peak": hb, "peak_source": src}), flush=True)
    lat.close()
    return 0


def run_persist_kernel(args, w):
    """Even-odd CG (FP32 inner, FP64 reliable updates) solved alone on 4^4,
    8^4, 12^4, 16^3x32 and 24^3x48 lattices (links exp(i 0.5 H), kappa 0.13,
    csw 1, Gaussian source): graph-replayed launch per stage against one
    persistent launch per iteration block; microseconds per iteration."""
    import torch

    import synth
    from paper_1103_1363_gb300 import lqcd
    stream = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for dims in ((4, 4, 4, 4), (8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 32), (24, 24, 24, 48)):
        lat = lqcd.Lattice(dims, precisions=("f64", "f32"), stream=stream)
        lat.gauge_load(torch.from_numpy(synth.smooth_gauge(dims, 0.5, 4)).cuda())
        lat.clover_compute(0.13, 1.0)
        b = torch.from_numpy(synth.gaussian_spinor(dims, 5)).cuda()
        x = torch.zeros_like(b)
        row = {"dims": list(dims)}
        for name, kw in (("graph", dict(use_graph=1)), ("persistent", dict(persistent=1))):
            best = None
            for rep in range(args.warmup + args.steps):
                stream.synchronize()
                e0.record(stream)
                rc, st = lat.solve(x, b, TOL, raise_on_error=False, inner_prec="f32", **kw)
                e1.record(stream)
                stream.synchronize()
                t = e0.elapsed_time(e1) * 1e-3
                if rep >= args.warmup and (best is None or t < best):
                    best = t
            row[name] = {"seconds": round(best, 5), "iterations": st["iterations"], "status": rc,
                         "us_per_iteration": round(1e6 * best / max(1, st["iterations"]), 2),
                         "true_residual": st["true_residual"], "launches": st["kernel_launches"]}
        print(json.dumps(row), flush=True)
        lat.close()
    return 0


def sap_block_flops(block):
    """FP32 flops per site and MR iteration of the SAP block solve: the
    block-restricted hops (165 each: projection, two SU(3) x vector products,
    reconstruction), the clover term (504), and the MR vector work (384:
    q = A rho - kappa h, |q|^2, <q, rho>, z += a rho, rho -= a q)."""
    hops = sum(2.0 * (b - 1) / b for b in block)
    return 165.0 * hops + 504.0 + 384.0


def run_sap_kernel(args, w):
    """SAP on the workload's lattice: the application z = SAP(r) alone
    (rotating buffers, larger than L2), then SAP-FGCR(24), SAP-FGMRES-DR
    (70 vectors, 10 deflated) and SAP-FGMRES(70) against identity-FGCR and
    the even-odd CG (FP16-spinor and all-FP16 inner) to the same tolerance."""
    import torch

    import synth
    from paper_1103_1363_gb300 import lqcd
    dims = w["dims"]
    V = int(np.prod(dims))
    block = tuple(int(b) for b in args.block.split("x"))
    K = 24
    MDR, KDR = 70, 10  # FGMRES-DR: Krylov space of 70 with 10 deflated vectors, as in Sec. 7
    stream = torch.cuda.Stream()
    lat = lqcd.Lattice(dims, precisions=("f64", "f32", "f16"), recon=12, gcr_nkrylov=MDR, stream=stream)
    lat.gauge_load(torch.from_numpy(synth.smooth_gauge(dims, w["eps"], w["gauge_seed"])).cuda())
    lat.clover_compute(w["kappa"], w["csw"])
    b = synth.gaussian_spinor(dims, w["src_seed"])
    nbuf = 4
    with torch.cuda.stream(stream):
        rs = [lat.new_field("f32", full=True) for _ in range(nbuf)]
        zs = [lat.new_field("f32", full=True) for _ in range(nbuf)]
    for f in rs:
        lat.pack(f, b, -1, "f32")
    for i in range(args.warmup):
        lat.sap_apply(zs[i % nbuf], rs[i % nbuf], block, args.ncycle, args.nmr)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        lat.sap_apply(zs[i % nbuf], rs[i % nbuf], block, args.ncycle, args.nmr)
    e1.record(stream)
    stream.synchronize()
    t = e0.elapsed_time(e1) * 1e-3 / args.steps
    fl = sap_block_flops(block) * args.nmr * args.ncycle * V
    pk = lqcd.lqcd_fma_peak(torch.cuda.current_device(), 0)
    out = {"kernel": "sap", "workload": workload_name(w), "block": list(block), "ncycle": args.ncycle,
           "nmr": args.nmr, "ms_per_application": round(t * 1e3, 3),
           "block_solve_flops_per_application": fl, "block_solve_gflops": round(fl / t / 1e9, 1),
           "fp32_peak_tflops": round(pk, 1), "alu_frac": round(fl / t / 1e12 / pk, 4)}
    del rs, zs
    if args.quick:
        print(json.dumps(out), flush=True)
        return 0
    bd = torch.from_numpy(b).cuda()
    xd = lat.canonical_spinor()
    solves = {}
    for name, sap, kw in (("fgcr_sap", True, dict(solver=lqcd.SOLVER_FGCR, inner_prec="f32", nkrylov=K)),
                          ("fgmres_dr_sap", True, dict(solver=lqcd.SOLVER_FGMRES_DR, inner_prec="f32", nkrylov=MDR,
                                                       ndefl=KDR)),
                          ("fgmres_sap", True, dict(solver=lqcd.SOLVER_FGMRES_DR, inner_prec="f32", nkrylov=MDR,
                                                    ndefl=0)),
                          ("eo_cg_f16spinors_inner", False, dict(inner_prec="f16spinors", reliable_interval=50,
                                                                 check_interval=10)),
                          ("eo_cg_f16_inner", False, dict(inner_prec="f16", reliable_interval=50,
                                                          check_interval=10)),
                          ("fgcr_identity", False, dict(solver=lqcd.SOLVER_FGCR, inner_prec="f32", nkrylov=K,
                                                        maxiter=20000)),
                          ("fgmres_dr_identity", False, dict(solver=lqcd.SOLVER_FGMRES_DR, inner_prec="f32",
                                                             nkrylov=MDR, ndefl=KDR, maxiter=20000)),
                          ("fgmres_identity", False, dict(solver=lqcd.SOLVER_FGMRES_DR, inner_prec="f32", nkrylov=MDR,
                                                          ndefl=0, maxiter=20000))):
        lat.set_sap(block if sap else None, args.ncycle, args.nmr)
        if not name.endswith("_identity"):
            lat.solve(xd, bd, TOL, raise_on_error=False, **kw)  # warm-up (graphs, first-touch)
        stream.synchronize()
        e0.record(stream)
        rc, st = lat.solve(xd, bd, TOL, raise_on_error=False, **kw)
        e1.record(stream)
        stream.synchronize()
        solves[name] = {"seconds": round(e0.elapsed_time(e1) * 1e-3, 4), "iterations": st["iterations"],
                        "true_residual": st["true_residual"], "status": rc,
                        "fallback": st["preconditioner_fallback"]}
    lat.set_sap(None)
    out["solves"] = solves
    print(json.dumps(out), flush=True)
    return 0


def bf16_peak():
    """Measured dense BF16 burst peak (TFLOP/s) and its source."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def run_net_kernel(args, w):
    """The BF16 parallel-transport network of the learned preconditioner on
    a 16^4 lattice (links exp(i 0.5 H), seed 100), widths 1 -> 12 -> 12 -> 1:
    the 3-layer forward at batch 1 (one preconditioner application), then at
    batch --batch the 12 -> 12 layer, its adjoint, its weight gradient and a
    whole training step.  Each is timed with CUDA events on the context's
    stream over --steps calls after --warmup; the library's kernel timer
    (lqcd_net_profile_*) gives the layer kernels' own device time, without
    the layout conversions at the ABI calls.  Inputs are seeded complex
    Gaussian activations."""
    import torch

    import synth
    from paper_1103_1363_gb300 import learned, lqcd
    dims = (16, 16, 16, 16)
    V = int(np.prod(dims))
    B = args.batch
    stream = torch.cuda.Stream()
    lat = lqcd.Lattice(dims, precisions=("f64", "f32"), stream=stream)
    lat.gauge_load(torch.from_numpy(synth.smooth_gauge(dims, 0.5, 100)).cuda())
    chans = (1, 12, 12, 1)
    net = lqcd.Net(lat, chans, bf16=True, max_batch=B)
    net.set_max_ctas(args.max_ctas)
    net.set_weights(learned.init_weights(chans, 7, scale=0.1))
    gen = torch.Generator().manual_seed(11)

    def act(ch, batch):
        return torch.randn((batch, V, ch, 4, 3), dtype=torch.complex64, generator=gen).to("cuda")

    x1, x12, g12 = act(1, B), act(12, B), act(12, B)
    y1, y12 = torch.empty_like(x1), torch.empty_like(x12)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pk, psrc = bf16_peak()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        stream.synchronize()
        net.profile_enable(True)
        net.profile_read()
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        stream.synchronize()
        prof = net.profile_read()
        net.profile_enable(False)
        return e0.elapsed_time(e1) / args.steps, prof

    out = {"kernel": "net", "workload": "parallel-transport network 1-12-12-1, BF16 tensor cores, 16^4, "
                                        "exp(i 0.5 H) links", "batch": B, "max_ctas": args.max_ctas,
           "peak_tflops": pk, "peak_source": psrc + " bf16 burst"}

    def kern(prof, key):
        e = prof[key]
        if e["launches"] == 0:
            return None
        us = 1e3 * e["ms"] / e["launches"]
        tf = e["flops"] / (e["ms"] * 1e-3) / 1e12
        return {"launches": e["launches"], "us_per_launch": round(us, 2), "tflops": round(tf, 1),
                "frac": round(tf / pk, 4), "achieved_gbs": round(e["bytes"] / (e["ms"] * 1e-3) / 1e9, 1)}

    ms, prof = timed(lambda: net.forward(y1[:1], x1[:1], 1))
    out["forward_batch1"] = {"ms_per_call": round(ms, 4),
                             "layers": {"%d" % l: kern(prof, (l, "fwd")) for l in range(3)}}
    ms, prof = timed(lambda: net.layer_apply(1, y12, x12, batch=B))
    out["layer12"] = dict(kern(prof, (1, "fwd")), ms_per_call_with_conversions=round(ms, 4))
    ms, prof = timed(lambda: net.layer_apply(1, y12, g12, batch=B, adjoint=True))
    out["layer12_adjoint"] = dict(kern(prof, (1, "adj")), ms_per_call_with_conversions=round(ms, 4))
    ms, prof = timed(lambda: net.layer_wgrad(1, x12, g12, batch=B))
    out["layer12_wgrad"] = dict(kern(prof, (1, "wgrad")), ms_per_call_with_conversions=round(ms, 4))
    r, e = act(1, B)[:, :, 0], act(1, B)[:, :, 0]
    r, e = r.contiguous(), e.contiguous()
    ms, prof = timed(lambda: net.train_step(r, e, B, lr=0.0))
    out["train_step"] = {"ms_per_step": round(ms, 4),
                         "kernels": {"%d_%s" % k: kern(prof, k) for k in prof if prof[k]["launches"]}}
    print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------------------ oracle (CPU)

def oracle_sample(w, napply):
    """The FP64 CPU oracle's Schur operator on the same lattice: napply
    applications (2 hopping terms each) timed on the host cores."""
    import oracle
    import synth
    dims = w["dims"]
    V = int(np.prod(dims))
    U = synth.smooth_gauge(dims, w["eps"], w["gauge_seed"])
    psi = synth.gaussian_spinor(dims, w["src_seed"])
    A = oracle.clover(U, w["kappa"], w["csw"])
    Ainv, _ = oracle.invert_site_matrices(A)
    oracle.schur(U, A, Ainv, w["kappa"], psi)  # touch memory once
    times = []
    for _ in range(napply):
        t0 = time.perf_counter()
        oracle.schur(U, A, Ainv, w["kappa"], psi)
        times.append(time.perf_counter() - t0)
    flops_per = 2 * 1320.0 * (V // 2)
    return {"times": times, "gflops": flops_per * len(times) / sum(times) / 1e9,
            "cores": oracle.num_threads()}


def oracle_solves():
    """The oracle's full solves on the host cores: 4^4 Haar (kappa 0.12, no
    clover) by CG on M^dag M and 16^3x32 (exp(i 0.5 H) links, kappa 0.135,
    csw 1) by even-odd CG, both to true residual 1e-10, on all cores and on
    one core; the one-core 16^3x32 solve runs 10 iterations and is
    extrapolated to the all-core run's iteration count (labelled)."""
    import oracle
    import synth
    cores = oracle.num_threads()
    out = {"cores_all": cores}
    d0 = (4, 4, 4, 4)
    U0, b0 = synth.haar_gauge(d0, 1), synth.gaussian_spinor(d0, 0)
    d1 = (16, 16, 16, 32)
    U1, b1 = synth.smooth_gauge(d1, 0.5, 2), synth.gaussian_spinor(d1, 0)
    t0 = time.perf_counter()
    A1 = oracle.clover(U1, 0.135, 1.0)
    A1inv, _ = oracle.invert_site_matrices(A1)
    out["c1_clover_setup_s"] = round(time.perf_counter() - t0, 3)
    try:
        for label, n in (("all_cores", cores), ("one_core", 1)):
            oracle.set_num_threads(n)
            t0 = time.perf_counter()
            _, it, res, ok = oracle.cgnr(U0, None, 0.12, b0)
            out["c0_4c4_cgnr_" + label] = {"seconds": round(time.perf_counter() - t0, 4), "iterations": it,
                                           "true_residual": res, "converged": ok, "threads": n}
        oracle.set_num_threads(cores)
        t0 = time.perf_counter()
        _, it, res, ok = oracle.eo_cg(U1, A1, A1inv, 0.135, b1)
        t_all = time.perf_counter() - t0
        out["c1_16c32_eo_cg_all_cores"] = {"seconds": round(t_all, 3), "iterations": it, "true_residual": res,
                                           "converged": ok, "threads": cores}
        oracle.set_num_threads(1)
        t0 = time.perf_counter()
        oracle.schur_cg_iters(U1, A1, A1inv, 0.135, b1, 10)
        t10 = time.perf_counter() - t0
        out["c1_16c32_eo_cg_one_core"] = {"seconds_per_iteration": round(t10 / 10, 4),
                                          "seconds_extrapolated": round(t10 / 10 * it, 2),
                                          "note": "10 iterations timed, extrapolated to %d" % it, "threads": 1}
    finally:
        oracle.set_num_threads(cores)
    return out


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    o = oracle_sample(w, args.warmup + args.steps)
    times = o["times"][args.warmup:]
    V = int(np.prod(w["dims"]))
    val = 2 * 1320.0 * (V // 2) * len(times) / sum(times) / 1e9
    sample = ("%d applications of the oracle's even-odd Schur operator (2 hopping terms each) on the "
              "full %s lattice, FP64, OpenMP" % (len(times), "x".join(map(str, w["dims"]))))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(w), "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": o["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="32c64", choices=sorted(WORKLOADS))
    ap.add_argument("--quick", action="store_true", help="skip the comparison legs (and the solves of --kernel sap)")
    ap.add_argument("--inner", default="f16spinors", choices=["f32", "f16", "bf16", "f16links", "bf16links", "f16spinors",
                                                      "bf16spinors"],
                    help="storage of the timed solve's inner iteration")
    ap.add_argument("--kernel", default=None, choices=["hop", "sap", "net", "persist"],
                    help="instead of the solve: time the stand-alone parity hopping kernel, the SAP "
                         "preconditioner and SAP-FGCR, or the learned preconditioner's network kernels "
                         "(profiling)")
    ap.add_argument("--batch", type=int, default=16, help="batch of --kernel net's layer and training timings")
    ap.add_argument("--max-ctas", type=int, default=0, help="CTA cap of --kernel net (0: one per SM)")
    ap.add_argument("--block", default="4x4x4x4", help="SAP block extents of --kernel sap")
    ap.add_argument("--ncycle", type=int, default=5, help="SAP cycles of --kernel sap")
    ap.add_argument("--nmr", type=int, default=4, help="MR iterations per block of --kernel sap")
    ap.add_argument("--prec", default="f16", help="precision of --kernel hop")
    ap.add_argument("--recon", type=int, default=12, choices=[12, 18], help="link storage of --kernel hop")
    ap.add_argument("--nrhs", type=int, default=1, help="right-hand sides per launch of --kernel hop")
    ap.add_argument("--staged", action="store_true",
                    help="--kernel hop: the shared-memory staged kernel (FP32 links, recon-12) instead of the gathering one")
    ap.add_argument("--cpu-applications", type=int, default=3)
    ap.add_argument("--skip-learned", action="store_true", help="leave out the learned-preconditioner leg")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    if args.kernel == "hop":
        return run_hop_kernel(args, w)
    if args.kernel == "sap":
        return run_sap_kernel(args, w)
    if args.kernel == "net":
        return run_net_kernel(args, w)
    if args.kernel == "persist":
        return run_persist_kernel(args, w)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    r = run_ours(args, w, rank, world, local_rank)
    if rank == 0:
        cpu = None
        if world == 1 and not args.quick:
            o = oracle_sample(w, args.cpu_applications)
            cpu = {"value": o["gflops"], "unit": "GFLOP/s", "cores": o["cores"], "kind": "oracle",
                   "sample": "%d applications of the oracle's even-odd Schur operator (2 hopping terms "
                             "each) on the full %s lattice, FP64, OpenMP on all host cores"
                             % (args.cpu_applications, "x".join(map(str, w["dims"]))),
                   "solves": oracle_solves()}
        ms_step = r["ms"] / args.steps
        line = {
            "metric": METRIC, "value": round(r["value"], 2), "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "storage": STORAGE[args.inner] + "; f64 reliable updates",
            "data": "synthetic",
            "config": {"workload": workload_name(w), "inner": args.inner, "reliable_update_every": RELIABLE_EVERY,
                       "reliable_delta": RELIABLE_DELTA,
                       "recon": 12, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (working set > 1 GB per solve)"},
            "roofline": r["roofline"], "cpu_baseline": cpu, "e2e": r.get("e2e"),
            "gpu_launches": r["launches"], "clocks": r["clocks"],
            "solve_per_step": {"iterations": r["stats"][-1]["iterations"],
                               "reliable_updates": r["stats"][-1]["reliable_updates"],
                               "dslash": r["stats"][-1]["dslash_count"],
                               "true_residual_max": r["worst_res"]},
            "clover_setup_s": r["clover_setup_s"], "tuned": r["tuned"],
            "solve": r.get("solve"), "dslash_f32": r.get("dslash_f32"), "alu_peaks": r.get("alu_peaks"),
            "multi_rhs": r.get("multi_rhs"), "learned": r.get("learned"),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
