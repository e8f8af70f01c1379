#!/usr/bin/env python
"""Benchmark of the hot path on synthetic inputs shaped like the paper's runs.

Workload (default): N = 2^20 points on a 1024 x 1024 jittered grid in [0,1]^2
(+-0.25 cell), Matern-1/2 with l = 0.1 (the paper's Table 1 kernel), rho = 3,
16 right-hand sides; Matern-3/2 is factored on the same pattern as well.
One step = maximin ordering -> pattern S_rho -> schedule -> ICHOL(0) in the
FP32 form -> solve L L^T x = b for the 16 right-hand sides, all on the GPU
with inputs already resident.  The FP64 factor (+ solve) is timed on the same
pattern for comparison.
Metric: nnz(L) per second of a whole step (and of the factor kernel, the
paper's t_ICHOL).  The default line also carries the rho = 2 and 5 patterns,
the sampled error estimator E of both factors, the supernodal block
factorisation, a refined solve to 1e-10, the 3-D configuration with its
rank-k PCA, the 256-set batched launch and a serving run.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs an
independent replica of the workload on its own GPU ("replicas only": a single
factor does not shard); value = nnz of all ranks / max over ranks of the time.
"""
from __future__ import annotations

import argparse
import itertools
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

from paper_1706_02205_gb300 import inputs  # noqa: E402

METRIC = "ICHOL(0) nnz(L)/s at N=2^20 d=2 rho=3, FP32-form vs FP64; serve p50/p99 ms"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def bytes_op(rowptr: np.ndarray, N: int, d: int, s: int) -> int:
    """Operand bytes of the left-looking factor with value size s:
    the pivot row staged once per column, the prefix of row j below i and x_j
    for every entry (j,i), the pattern read and L written once, the points
    read once.  sum over (j,i) of |R_j cap [0,i)| = sum_j |R_j|(|R_j|-1)/2."""
    r = np.diff(rowptr).astype(np.int64) - 1
    rsum = int(r.sum())
    pre = int((r * (r - 1) // 2).sum())
    nnz = int(rowptr[-1])
    return rsum * (4 + s) + pre * (4 + s) + (nnz - N) * 8 * d + nnz * (4 + s) + N * d * 8


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, dev_index: int):
        self.f = tempfile.NamedTemporaryFile(prefix="clk", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev_index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.f.name):
            c = [v.strip() for v in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            for nm, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- our arm

def run_ours(args, rank, world):
    import torch

    from paper_1706_02205_gb300 import kchol as kc

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    x_h = inputs.jittered_grid(args.n_side, seed=inputs.seed_for(2, rank))
    N, d = x_h.shape
    b_h = inputs.rhs(N, args.nrhs, seed=inputs.seed_for(2, 100 + rank))
    kern = kc.Kernel(args.nu, args.ell, 1.0, 0.0)
    x = torch.from_numpy(x_h).to(dev)
    b = torch.from_numpy(b_h).to(dev)
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step(prec=kc.FP32_FORM, ev=None):
        if ev:
            ev[0].record(stream)
        perm, l, xo = kc.order_points(x)
        if ev:
            ev[1].record(stream)
        rowptr, col = kc.pattern_rows(xo, l, args.rho)
        if ev:
            ev[2].record(stream)
        pat = kc.schedule(rowptr, col, xo)
        if ev:
            ev[3].record(stream)
        val, diag, zp = kc.factor(pat, xo, kern, prec)
        if ev:
            ev[4].record(stream)
        xs = kc.solve(pat, prec, val, diag, kern, perm, b)
        if ev:
            ev[5].record(stream)
        return dict(perm=perm, l=l, xo=xo, pat=pat, val=val, diag=diag, zp=zp, xs=xs)

    from paper_1706_02205_gb300 import replicas
    barrier = replicas.barrier

    for _ in range(args.warmup):
        r = step()
    torch.cuda.synchronize()
    pat = r["pat"]
    nnz = pat.nnz
    rowptr_h = pat.rowptr.cpu().numpy()

    names = ["order", "pattern", "schedule", "factor", "solve"]
    phase = {n: [] for n in names}
    step_ms, fk_ms = [], []
    launches0 = kc.launch_count()
    clk = Clocks(dev.index) if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        r = step(kc.FP32_FORM, ev)
        torch.cuda.synchronize()
        fk_ms.append(kc.last_factor_kernel_ms())
        for k, n in enumerate(names):
            phase[n].append(ev[k].elapsed_time(ev[k + 1]))
        step_ms.append(ev[0].elapsed_time(ev[5]))
    torch.cuda.synchronize()
    barrier()
    launches = kc.launch_count() - launches0
    clocks = clk.stop() if clk else None

    # FP64 factor + solve on the same pattern (plain-method comparison)
    pat, xo, perm = r["pat"], r["xo"], r["perm"]
    f64_ms, f64_k, s64_ms = [], [], []
    for it in range(args.warmup + args.steps):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        v64, d64, zp64 = kc.factor(pat, xo, kern, kc.FP64)
        e[1].record(stream)
        kc.solve(pat, kc.FP64, v64, d64, kern, perm, b)
        e[2].record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            f64_ms.append(e[0].elapsed_time(e[1]))
            s64_ms.append(e[1].elapsed_time(e[2]))
            f64_k.append(kc.last_factor_kernel_ms())

    # the paper's accuracy measure (Section 4.4) of both headline factors: the
    # sampled estimator E over 500,000 uniform index pairs, 50 repetitions
    # (mean and standard deviation, as the paper reports it)
    accuracy = {}
    for pname, pr, vv, dd in (("fp32_form", kc.FP32_FORM, r["val"], r["diag"]), ("fp64", kc.FP64, v64, d64)):
        es = []
        for rep in range(args.e_reps):
            pi_h, pj_h = inputs.sample_pairs(N, 500_000, seed=inputs.seed_for(2, 200 + rep))
            n2, d2, _ = kc.frob_error(pat, pr, vv, dd, xo, kern, perm, torch.from_numpy(pi_h).to(dev),
                                      torch.from_numpy(pj_h).to(dev))
            es.append((n2 / d2) ** 0.5)
        accuracy[pname] = {"E_mean": statistics.mean(es), "E_std": statistics.pstdev(es), "repetitions": len(es),
                           "pairs_per_repetition": 500_000}

    # the other kernel of the workload on the same pattern (the pattern does not
    # depend on the kernel): factor only, both precisions
    other = {}
    for nu2 in args.other_nu:
        k2 = kc.Kernel(nu2, args.ell, 1.0, 0.0)
        res = {}
        for pname, pr in (("fp32_form", kc.FP32_FORM), ("fp64", kc.FP64)):
            ks, zps = [], []
            for it in range(1 + args.steps):
                flush.zero_()
                _, _, zz = kc.factor(pat, xo, k2, pr)
                torch.cuda.synchronize()
                if it >= 1:
                    ks.append(kc.last_factor_kernel_ms())
                    zps.append(zz)
            res[pname] = {"kernel_ms": statistics.mean(ks), "kernel_nnz_per_s": nnz / (statistics.mean(ks) * 1e-3),
                          "zero_pivots": zps[-1]}
        other[f"matern_nu{nu2}"] = res

    # rho = 2 and 5 (the other patterns of the configuration): ordering and
    # pattern once, then each factor kernel timed after one warm-up
    rho_sweep = {}
    for rho2 in args.other_rho:
        p2 = kc.build_pattern(xo, r["l"], rho2)
        ent = {"nnz": p2.nnz, "depth": p2.depth}
        for nu2 in [args.nu] + list(args.other_nu):
            k2 = kc.Kernel(nu2, args.ell, 1.0, 0.0)
            for pname, pr in (("fp32_form", kc.FP32_FORM), ("fp64", kc.FP64)):
                ks = []
                for it in range(1 + max(1, args.steps // 2)):
                    flush.zero_()
                    _, _, zz = kc.factor(p2, xo, k2, pr)
                    torch.cuda.synchronize()
                    if it >= 1:
                        ks.append(kc.last_factor_kernel_ms())
                km = statistics.mean(ks)
                ent[f"matern_nu{nu2}_{pname}"] = {"kernel_ms": km, "kernel_nnz_per_s": p2.nnz / (km * 1e-3),
                                                  "zero_pivots": zz}
        rho_sweep[f"rho{rho2:g}"] = ent
        del p2

    # end to end through the public calls from pinned host buffers
    xp = torch.from_numpy(x_h).pin_memory()
    bp = torch.from_numpy(b_h).pin_memory()
    out = torch.empty((args.nrhs, N), dtype=torch.float64).pin_memory()
    e2e_ms = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xd = xp.to(dev, non_blocking=True)
        bd = bp.to(dev, non_blocking=True)
        perm_, l_, xo_ = kc.order_points(xd)
        pat_ = kc.build_pattern(xo_, l_, args.rho)
        val_, diag_, _ = kc.factor(pat_, xo_, kern, kc.FP32_FORM)
        xs_ = kc.solve(pat_, kc.FP32_FORM, val_, diag_, kern, perm_, bd)
        out.copy_(xs_, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        del pat_, val_, diag_, xs_

    # max over ranks
    tot_ms, e2e_tot = replicas.max_over_ranks([sum(step_ms), sum(e2e_ms)], device=dev)

    if rank != 0:
        return None
    hbm, peak_kind = peaks()
    bop = bytes_op(rowptr_h, N, d, 4)
    ns = 1 << max(0, (args.nrhs - 1).bit_length())
    fk = statistics.mean(fk_ms)
    achieved = bop / (fk * 1e-3) / 1e9
    value = world * nnz * args.steps / (tot_ms * 1e-3)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "nnz(L)/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 values + f64 pivots (FP32 form)",
        "data": "synthetic",
        "config": {"workload": f"jittered grid {args.n_side}x{args.n_side} (N={N}) in [0,1]^2, Matern-{args.nu} "
                               f"l={args.ell}, rho={args.rho}, {args.nrhs} rhs; step = order+pattern+schedule+"
                               f"factor(FP32 form)+solve",
                   "N": N, "d": d, "nnz": nnz, "nnz_per_row": nnz / N, "depth": pat.depth,
                   "zero_pivots": r["zp"], "l2": "working set > L2 (GBs); 256 MB L2 flush between steps",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "phases_ms": {n: statistics.mean(v) for n, v in phase.items()},
        "factor_fp32_form": {"nnz_per_s": nnz / (statistics.mean(phase["factor"]) * 1e-3),
                             "kernel_ms": fk, "kernel_nnz_per_s": nnz / (fk * 1e-3)},
        "factor_fp64": {"nnz_per_s": nnz / (statistics.mean(f64_ms) * 1e-3), "call_ms": statistics.mean(f64_ms),
                        "kernel_ms": statistics.mean(f64_k), "solve_ms": statistics.mean(s64_ms)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": args.traffic if args.traffic is not None else factor_traffic(bop),
                     "peak_kind": f"{peak_kind} hbm_gbs (burst)",
                     "kernel": "ichol_persistent_k<float>", "algorithmic_bytes": bop},
        "e2e": {"value": world * nnz * max(1, args.steps) / (e2e_tot * 1e-3), "unit": "nnz(L)/s",
                "ms_per_step": e2e_tot / max(1, args.steps),
                "h2d_bytes_per_step": int(x_h.nbytes + b_h.nbytes), "d2h_bytes_per_step": int(out.numel() * 8)},
        "other_kernels_same_pattern": other,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    # the triangular solves: compulsory bytes (pattern and L read once
    # per direction, the right-hand sides in and out) over their time
    solve_bytes = (nnz * 8 + (N + 1) * 8) + (nnz * 16 + (N + 1) * 8) + 4 * N * ns * 8 + 2 * N * args.nrhs * 8
    solve_ms = statistics.mean(phase["solve"])
    line["solve_roofline"] = {"bound": "latency (dependency depth x row latency)", "algorithmic_bytes": solve_bytes,
                              "achieved": solve_bytes / (solve_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                              "frac": solve_bytes / (solve_ms * 1e-3) / 1e9 / hbm, "ms": solve_ms,
                              "kernels": "fwd_solve_pair_k<16> + bwd_solve_pair_k<16> + permutations"}
    line["rho_sweep"] = rho_sweep
    line["accuracy_E"] = accuracy
    if args.supernodal_leg:
        line["supernodal"] = supernodal_leg(args, r["l"], xo, pat, kern)
    if args.refine_side > 0:
        line["refine_to_1e-10"] = run_refine(args)
    if args.config_legs and world == 1:
        # the 3-D configuration (factor, rank-k PCA and its error) and the 256-set batched launch
        small = argparse.Namespace(**dict(vars(args), steps=2, warmup=1))
        line["config3_cube3d"] = run_cube3d(small)
        line["config4_batch"] = run_batch(small)
    if args.serve_leg:
        from paper_1706_02205_gb300 import serve
        args.serve_fracs = (0.8,)
        line["serve"] = serve.bench(args)
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    return line


# ------------------------------------------------ other workloads (ours)

def supernodal_leg(args, l, xo, pat0, kern):
    """The supernodal multicolour ordering and pattern built from the headline
    step's maximin order and pattern, and the block factorisation on it (both
    forms) beside the column-task kernel on the same pattern; kernel times
    from CUDA events, median of the timed runs after one warm-up."""
    import torch

    from paper_1706_02205_gb300 import kchol as kc
    stream = torch.cuda.current_stream()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    sn = kc.supernodal(xo, l, args.rho, pat0, with_schedule=False)
    e[1].record(stream)
    spat = kc.schedule(sn["rowptr"], sn["col"], sn["x_new"])
    e[2].record(stream)
    torch.cuda.synchronize()
    out = {"construction_ms": e[0].elapsed_time(e[1]), "schedule_ms": e[1].elapsed_time(e[2]), "nnz": spat.nnz,
           "depth": spat.depth}
    xn = sn["x_new"]
    for name, fn, pr in (("blocked_fp32_form", kc.factor_blocked, kc.FP32_FORM),
                         ("blocked_fp64", kc.factor_blocked, kc.FP64),
                         ("column_fp32_form", kc.factor, kc.FP32_FORM)):
        ks, cs = [], []
        for it in range(1 + max(1, args.steps // 2)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, zp = fn(spat, xn, kern, pr)
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= 1:
                ks.append(kc.last_factor_kernel_ms())
                cs.append(e0.elapsed_time(e1))
        km = statistics.median(ks)
        # call_ms: the whole call (the blocked factor's group detection and task list included)
        out[name] = {"kernel_ms": km, "kernel_nnz_per_s": spat.nnz / (km * 1e-3), "zero_pivots": zp,
                     "call_ms": statistics.median(cs)}
    return out


# DRAM traffic of the FP32-form factor kernel per algorithmic byte, from the ncu capture of the factor
# on the 512x512 jittered grid (dram read + write = 28.119 GB for
# B_op = 26.388 GB).  Both are sums over the same (j, i) pairs, so the ratio carries to the full size.
# It is reported only while the kernel's sources are the ones the counters were taken on (the
# interface header adds only the struct layouts, which tests/test_abi.py pins field by field).
TRAFFIC_CAPTURE = {"sources": ("paper_1706_02205_gb300/csrc/factor.cu", "paper_1706_02205_gb300/csrc/common.cuh",
                               "paper_1706_02205_gb300/csrc/grid.cuh", "paper_1706_02205_gb300/csrc/covariance.cuh",
                               "paper_1706_02205_gb300/csrc/ichol.cuh"),
                   "sha256": "c5116e557deef04bec67567413686605b69b2985ad7105fa046902e1ceec735f",
                   "dram_per_algorithmic_byte": (27.158938 + 0.959845) / 26.387813}


def factor_traffic(bop):
    """ncu DRAM bytes per factor launch scaled from the capture, or None if the kernel changed since."""
    import hashlib
    h = hashlib.sha256()
    try:
        for rel in TRAFFIC_CAPTURE["sources"]:
            with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), rel), "rb") as f:
                h.update(f.read())
    except OSError:
        return None
    if h.hexdigest() != TRAFFIC_CAPTURE["sha256"]:
        return None
    return TRAFFIC_CAPTURE["dram_per_algorithmic_byte"] * bop


def make_kernel(args):
    """The covariance function the options name (--family, --nu, --ell, --alpha, --beta)."""
    from paper_1706_02205_gb300 import kchol as kc
    if args.family == "cauchy":
        return kc.Kernel(ell=args.ell, family=kc.CAUCHY, alpha=args.alpha, beta=args.beta)
    return kc.Kernel(args.nu, args.ell)


def kernel_name(k):
    if k.family == 1:
        return f"Cauchy l={k.ell} alpha={k.alpha} beta={k.beta}"
    return f"Matern-{k.nu} l={k.ell}" + (f" nugget {k.nugget}" if k.nugget else "")


def run_tasks(args):
    """Tasks (1), (3), (4) with the factor on the 1024 x 1024 jittered grid
    (rho = 3, FP32 form): L L^T v for 16 and 1 vectors, one sample L z, and
    log det.  Each call includes its permutations to and from the original
    order; times are CUDA events around the call after warm-up."""
    import torch

    from paper_1706_02205_gb300 import kchol as kc
    x = torch.from_numpy(inputs.jittered_grid(args.n_side, seed=inputs.seed_for(2))).cuda()
    kern = make_kernel(args)
    perm, l, xo = kc.order_points(x)
    pat = kc.build_pattern(xo, l, args.rho)
    val, diag, zp = kc.factor(pat, xo, kern, kc.FP32_FORM)
    N, nnz, s = pat.N, pat.nnz, 4
    v16 = torch.from_numpy(inputs.rhs(N, 16, seed=inputs.seed_for(2, 70))).cuda()
    v1 = v16[:1].contiguous()
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ms = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    # algorithmic bytes: L pass = rowptr, col and val once, diag, the vectors in
    # and out once; L^T pass = colptr, rowidx, slot and val once, diag, the
    # vectors; the permutations read and write each vector once more
    def bytes_l(ns):
        return (N + 1) * 8 + nnz * (4 + s) + N * 8 + 2 * N * ns * 8

    def bytes_lt(ns):
        return (N + 1) * 8 + nnz * (4 + 8 + s) + N * 8 + 2 * N * ns * 8

    def bytes_perm(nrhs, ns):
        return 2 * (N * nrhs * 8 + N * ns * 8 + N * 4)

    out = {"workload": f"tasks on jittered grid {args.n_side}x{args.n_side} (N={N}), {kernel_name(kern)}, "
                       f"rho={args.rho}, FP32 form", "N": N, "nnz": nnz, "zero_pivots": zp, "calls": {}}
    for name, fn, b in (
            ("llt_matvec_16", lambda: kc.llt_matvec(pat, kc.FP32_FORM, val, diag, perm, v16),
             bytes_l(16) + bytes_lt(16) + bytes_perm(16, 16)),
            ("llt_matvec_1", lambda: kc.llt_matvec(pat, kc.FP32_FORM, val, diag, perm, v1),
             bytes_l(1) + bytes_lt(1) + bytes_perm(1, 1)),
            ("sample_l_matvec_1", lambda: kc.l_matvec(pat, kc.FP32_FORM, val, diag, perm, v1),
             bytes_l(1) + bytes_perm(1, 1)),
            ("lt_matvec_1", lambda: kc.lt_matvec(pat, kc.FP32_FORM, val, diag, perm, v1),
             bytes_lt(1) + bytes_perm(1, 1)),
            ("logdet", lambda: kc.logdet(pat, diag), N * 8)):
        ms = timed(fn)
        out["calls"][name] = {"ms": ms, "algorithmic_bytes": b, "GB_per_s": b / (ms * 1e-3) / 1e9}
    return out


def run_pde(args):
    """Section 6: the rough-coefficient grid operator (5-point stencil, edge
    weights log-uniform in [1/10, 10], plus --shift times the identity; the
    default 100 = 1/l^2 for the range l = 0.1 of the headline kernel) on the
    n_side x n_side grid, standing in for a precision matrix A = Theta^{-1}: maximin
    order, min-rule pattern, reversed, A gathered onto it, FP32-form factor,
    one solve.  Phases timed with CUDA events after warm-up; the residual
    ||A x - b|| / ||b|| of the approximate direct solve is measured outside."""
    import torch

    from paper_1706_02205_gb300 import kchol as kc
    n = args.n_side
    x_h, rp_h, col_h, val_h = inputs.grid_operator(n, shift=args.shift)
    x = torch.from_numpy(x_h).cuda()
    rp, col, val = (torch.from_numpy(a).cuda() for a in (rp_h, col_h, val_h))
    N = n * n
    b = torch.from_numpy(inputs.rhs(N, 1, seed=inputs.seed_for(6, 2))).cuda()
    dmax = float(val_h.max())
    stream = torch.cuda.current_stream()
    names = ("order", "pattern", "reverse", "gather", "factor", "solve")
    ph = {k: [] for k in names}
    for it in range(args.warmup + args.steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        ev[0].record(stream)
        perm, l, xo = kc.order_points(x)
        ev[1].record(stream)
        pat = kc.build_pattern(xo, l, args.rho, kc.RULE_MIN)
        ev[2].record(stream)
        rpat = kc.pattern_reverse(pat, xo)
        orig = perm.flip(0).contiguous()
        ev[3].record(stream)
        aval, _ = kc.gather_entries(rpat, orig, rp, col, val, count_outside=False)
        ev[4].record(stream)
        v, dg, zp = kc.factor_given(rpat, aval, kc.FP32_FORM)
        ev[5].record(stream)
        xs = kc.solve(rpat, kc.FP32_FORM, v, dg, kc.Kernel(sigma2=dmax), orig, b)
        ev[6].record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            for k, nm in enumerate(names):
                ph[nm].append(ev[k].elapsed_time(ev[k + 1]))
    _, outside = kc.gather_entries(rpat, orig, rp, col, val)
    A = torch.sparse_csr_tensor(rp, col.long(), val, size=(N, N))
    res = float(torch.linalg.vector_norm(A @ xs[0] - b[0]) / torch.linalg.vector_norm(b[0]))
    # CG on A preconditioned by the factor, to 1e-10
    cg = []
    for it in range(args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xr, iters, rr, st = kc.refine_sparse(rpat, kc.FP32_FORM, v, dg, orig, rp, col, val, b, rtol=1e-10,
                                             maxit=500)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            cg.append(e0.elapsed_time(e1))
    cg_res = float(torch.linalg.vector_norm(A @ xr[0] - b[0]) / torch.linalg.vector_norm(b[0]))
    med = {k: statistics.median(v_) for k, v_ in ph.items()}
    return {"workload": f"grid operator {n}x{n} (N={N}), rough coefficients, shift {args.shift}, reverse "
                        f"maximin order, min-rule rho={args.rho}, FP32 form", "N": N, "nnz": rpat.nnz, "depth": rpat.depth,
            "zero_pivots": zp, "entries_outside_pattern": outside, "phases_ms": med,
            "total_ms": sum(med.values()), "factor_nnz_per_s": rpat.nnz / (med["factor"] * 1e-3),
            "factor_kernel_ms": kc.last_factor_kernel_ms(), "direct_solve_relres": res,
            "cg_to_1e-10": {"ms": statistics.median(cg), "iterations": iters, "status": st,
                            "true_relres": cg_res}}


def run_supernodal(args):
    """The supernodal multicolour ordering and pattern on the 1024 x 1024
    jittered grid (rho, kernel as for the headline), FP32 form: the maximin
    order and max-rule pattern it starts from, the construction, the new
    pattern's schedule and the factor; phases by CUDA events after warm-up,
    with the maximin factor on the same points beside it."""
    import torch

    from paper_1706_02205_gb300 import kchol as kc
    x = torch.from_numpy(inputs.jittered_grid(args.n_side, seed=inputs.seed_for(2))).cuda()
    kern = make_kernel(args)
    stream = torch.cuda.current_stream()
    names = ("order", "pattern", "schedule", "supernodal", "schedule_new", "factor")
    ph = {k: [] for k in names}
    for it in range(args.warmup + args.steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        ev[0].record(stream)
        perm0, l, xo = kc.order_points(x)
        ev[1].record(stream)
        rowptr, col = kc.pattern_rows(xo, l, args.rho)
        ev[2].record(stream)
        pat0 = kc.schedule(rowptr, col, xo)
        ev[3].record(stream)
        N, d = xo.shape
        sn = kc.supernodal(xo, l, args.rho, pat0, with_schedule=False)
        rp, cl, x_new = sn["rowptr"], sn["col"], sn["x_new"]
        ev[4].record(stream)
        spat = kc.schedule(rp, cl, x_new)
        ev[5].record(stream)
        val, diag, zp = kc.factor(spat, x_new, kern, kc.FP32_FORM)
        ev[6].record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            for k, nm in enumerate(names):
                ph[nm].append(ev[k].elapsed_time(ev[k + 1]))
    sn_factor_kernel = kc.last_factor_kernel_ms()
    # the same pattern by column groups (the block factorisation), both forms
    blocked = {}
    for pname, pr in (("fp32_form", kc.FP32_FORM), ("fp64", kc.FP64)):
        ks, cs = [], []
        for it in range(args.warmup + args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            vb, db, zb = kc.factor_blocked(spat, x_new, kern, pr)
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= args.warmup:
                ks.append(kc.last_factor_kernel_ms())
                cs.append(e0.elapsed_time(e1))
        km = statistics.median(ks)
        blocked[pname] = {"kernel_ms": km, "kernel_nnz_per_s": spat.nnz / (km * 1e-3), "zero_pivots": zb,
                          "call_ms": statistics.median(cs)}
        del vb, db
    ks64 = []
    for it in range(1 + args.steps):
        kc.factor(spat, x_new, kern, kc.FP64)
        torch.cuda.synchronize()
        if it >= 1:
            ks64.append(kc.last_factor_kernel_ms())
    _, _, zp0 = kc.factor(pat0, xo, kern, kc.FP32_FORM)
    mm_factor_kernel = kc.last_factor_kernel_ms()
    med = {k: statistics.median(v_) for k, v_ in ph.items()}
    return {"workload": f"supernodal multicolour order, jittered grid {args.n_side}x{args.n_side} (N={N}), "
                        f"{kernel_name(kern)}, rho={args.rho}, FP32 form", "N": N, "nnz": spat.nnz,
            "depth": spat.depth, "zero_pivots": zp, "phases_ms": med,
            "factor_kernel_ms": sn_factor_kernel, "factor_nnz_per_s": spat.nnz / (sn_factor_kernel * 1e-3),
            "factor_fp64_kernel_ms": statistics.median(ks64), "blocked": blocked,
            "maximin": {"nnz": pat0.nnz, "depth": pat0.depth, "factor_kernel_ms": mm_factor_kernel,
                        "zero_pivots": zp0}}


def run_factor_only(args):
    """Factor-only probe (the launch profiled by ncu): order + pattern once,
    then the FP32-form factor `--steps` times on the same pattern."""
    import torch

    from paper_1706_02205_gb300 import kchol as kc
    if args.geom == "cube3d":  # the 3-D configuration: 2^18 uniform points, Matern-5/2 l=0.3, nugget, rho=4
        x = torch.from_numpy(inputs.uniform(args.n3, 3, seed=inputs.seed_for(3))).cuda()
        kern, rho = kc.Kernel(2.5, 0.3, 1.0, 1e-6), 4.0
    else:
        x = torch.from_numpy(inputs.jittered_grid(args.n_side, seed=inputs.seed_for(2))).cuda()
        kern, rho = make_kernel(args), args.rho
    perm, l, xo = kc.order_points(x)
    pat = kc.build_pattern(xo, l, rho)
    prec = kc.FP64 if args.prec == "fp64" else kc.FP32_FORM
    out = {"workload": f"factor-only {args.geom}", "kernel": kernel_name(kern), "N": pat.N, "nnz": pat.nnz, "depth": pat.depth, "prec": args.prec,
           "algorithmic_bytes": bytes_op(pat.rowptr.cpu().numpy(), pat.N, x.shape[1], 8 if args.prec == "fp64" else 4),
           "runs": []}
    for rpt, lanes, unroll, adapt, stage, warps in itertools.product(args.rpt, args.lanes, args.unroll, args.adaptive,
                                                                     args.stage, args.warps):
        o = kc.make_opts(rows_per_task=rpt, lanes_per_row=lanes, unroll=unroll, adaptive_chunks=adapt,
                         stage_bytes=stage, warps_per_cta=warps)
        ms = []
        for _ in range(args.steps):
            _, _, zp = kc.factor(pat, xo, kern, prec, o)
            torch.cuda.synchronize()
            ms.append(kc.last_factor_kernel_ms())
        out["runs"].append({"rpt": rpt, "lanes": lanes, "unroll": unroll, "adaptive": adapt, "stage": stage,
                            "warps": warps, "kernel_ms": min(ms), "zero_pivots": zp})
    return out


def run_cube3d(args):
    """N = 2^18 points uniform in [0,1]^3, Matern-5/2, l = 0.3, nugget 1e-6,
    rho = 4, FP32 form; rank-k PCA for k in {64, 512} with the operator-norm
    error from 50 power iterations."""
    import torch

    from paper_1706_02205_gb300 import kchol as kc
    N = args.n3
    x_h = inputs.uniform(N, 3, seed=inputs.seed_for(3))
    x = torch.from_numpy(x_h).cuda()
    kern = kc.Kernel(2.5, 0.3, 1.0, 1e-6)
    stream = torch.cuda.current_stream()
    ph = {k: [] for k in ("order", "pattern", "schedule", "factor", "pca64", "pca512")}
    for it in range(args.warmup + args.steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
        ev[0].record(stream)
        perm, l, xo = kc.order_points(x)
        ev[1].record(stream)
        rowptr, col = kc.pattern_rows(xo, l, 4.0)
        ev[2].record(stream)
        pat = kc.schedule(rowptr, col, xo)
        ev[3].record(stream)
        val, diag, zp = kc.factor(pat, xo, kern, kc.FP32_FORM)
        ev[4].record(stream)
        L64 = kc.pca_truncate(pat, kc.FP32_FORM, val, perm, 64)
        ev[5].record(stream)
        L512 = kc.pca_truncate(pat, kc.FP32_FORM, val, perm, 512)
        ev[6].record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            for k, n in enumerate(ph):
                ph[n].append(ev[k].elapsed_time(ev[k + 1]))
    v0 = torch.from_numpy(inputs.unit_vector(N, seed=inputs.seed_for(3, 9))).cuda()
    t0 = time.perf_counter()
    e64 = kc.pca_error(x, kern, L64, v0, iters=50)
    t1 = time.perf_counter()
    e512 = kc.pca_error(x, kern, L512, v0, iters=50)
    t2 = time.perf_counter()
    e0 = kc.pca_error(x, kern, L64[:0], v0, iters=50)  # ||Theta||_2 for scale
    fk = statistics.mean(ph["factor"])
    nnz = pat.nnz
    return {"workload": f"uniform [0,1]^3, N={N}, Matern-5/2 l=0.3 nugget 1e-6, rho=4, FP32 form",
            "N": N, "nnz": nnz, "nnz_per_row": nnz / N, "depth": pat.depth, "zero_pivots": zp,
            "phases_ms": {k: statistics.mean(v) for k, v in ph.items()},
            "factor_nnz_per_s": nnz / (fk * 1e-3), "factor_kernel_ms": kc.last_factor_kernel_ms(),
            "pca": {"theta_norm2_est": e0, "err_k64": e64, "err_k512": e512,
                    "rel_err_k64": e64 / e0, "rel_err_k512": e512 / e0,
                    "power_iter_s": {"k64": t1 - t0, "k512": t2 - t1}, "iters": 50}}


def run_batch(args):
    """256 independent sets, N_s log-uniform in [2000, 50000], 192 in 2-D and
    64 in 3-D, Matern-3/2 with l_s ~ U[0.05, 0.3], rho = 3, FP32 form: one
    persistent launch over all sets, tuned, recorded in a CUDA graph and
    replayed; plus one solve of every set at once."""
    import torch

    from paper_1706_02205_gb300 import batch as kb
    from paper_1706_02205_gb300 import kchol as kc
    from paper_1706_02205_gb300 import replicas
    rank, world = replicas.rank_world()
    sets = inputs.batch_sets(n_sets=args.n_sets)
    if world > 1:  # independent sets: split by size (the factor's work grows with N), no collective
        sets = [sets[i] for i in replicas.partition([s["x"].shape[0] for s in sets], world)[rank]]
    xs = [torch.from_numpy(s["x"]).cuda() for s in sets]
    kerns = [kc.Kernel(1.5, s["ell"]) for s in sets]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B = kb.BatchFactor(xs, kerns, 3.0, kc.FP32_FORM, n_streams=8)
    torch.cuda.synchronize()
    t_prep = time.perf_counter() - t0
    tuned = B.tune()
    B.capture()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        B.replay()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    zp = B.plan.finish()
    Ntot = sum(B.Ns)
    b = torch.from_numpy(inputs.rhs(Ntot, 1, seed=inputs.seed_for(4, 2))).cuda()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    B.solve(b)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t1
    # parity of a few sets against the same sets factored alone
    worst = 0.0
    for s in (0, len(sets) // 2, len(sets) - 1):
        r = kc.pipeline(xs[s], 3.0, kerns[s], kc.FP32_FORM,
                        opts=kc.make_opts(lanes_per_row=tuned["lanes_per_row"], unroll=tuned["unroll"]))
        worst = max(worst, float((B.set_values(s) - r["val"]).abs().max()))
    m = statistics.mean(ms)
    if world > 1:
        m_all = replicas.max_over_ranks([m])[0]
        nnz_all = replicas.sum_over_ranks([B.pat.nnz])[0]
        if rank != 0:
            return None
        return {"workload": f"{args.n_sets} sets split over {world} ranks by size, one graph-replayed launch each",
                "n_gpus": world, "graph_launch_ms_max": m_all, "aggregate_nnz_per_s": nnz_all / (m_all * 1e-3),
                "scaling": "weak"}
    return {"workload": f"{len(sets)} sets, N_s log-U[2000,50000] (sum N={Ntot}), 2-D/3-D, Matern-3/2 "
                        f"l_s~U[0.05,0.3], rho=3, FP32 form, one graph-replayed launch",
            "sets": len(sets), "N_total": Ntot, "nnz": B.pat.nnz, "depth": B.pat.depth, "zero_pivots": zp,
            "graph_launch_ms": m, "aggregate_nnz_per_s": B.pat.nnz / (m * 1e-3), "tuned": tuned,
            "prepare_s": t_prep, "solve_all_ms": t_solve * 1e3, "max_abs_diff_vs_alone": worst}


def run_refine(args):
    """Time to a refined solve (task (2)): factor (FP32 form or FP64) + CG on the
    dense Theta preconditioned by the factor, 16 right-hand sides to relative
    residual 1e-10, on the jittered grid of side --refine-side (the dense FP64
    product is O(N^2) per iteration: 2^16 points take about half a second per
    iteration on the GB300, whose FP64 pipe is a small fraction of its FP32
    rate, so 2^20 points would take over two minutes per iteration).  Each
    form: one warm-up, then the factor and the CG timed on the device (the CG
    synchronises every iteration for its convergence test)."""
    import torch

    from paper_1706_02205_gb300 import kchol as kc
    n = args.refine_side
    x = torch.from_numpy(inputs.jittered_grid(n, seed=inputs.seed_for(2, 30))).cuda()
    b = torch.from_numpy(inputs.rhs(n * n, args.nrhs, seed=inputs.seed_for(2, 31))).cuda()
    kern = kc.Kernel(args.nu, args.ell)
    perm, l, xo = kc.order_points(x)
    pat = kc.build_pattern(xo, l, args.rho)
    out = {"workload": f"jittered grid {n}x{n} (N={n * n}), Matern-{args.nu} l={args.ell}, rho={args.rho}, "
                       f"{args.nrhs} rhs, CG on the dense Theta (FP64) preconditioned by the factor, to 1e-10",
           "N": n * n, "nnz": pat.nnz}
    for name, prec in (("fp32_form", kc.FP32_FORM), ("fp64", kc.FP64)):
        kc.factor(pat, xo, kern, prec)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        val, diag, zp = kc.factor(pat, xo, kern, prec)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        xs, it, rr, st = kc.refine(pat, xo, kern, prec, val, diag, perm, b, rtol=1e-10, maxit=500)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out[name] = {"factor_ms": (t1 - t0) * 1e3, "refine_ms": (t2 - t1) * 1e3, "time_to_1e-10_ms": (t2 - t0) * 1e3,
                     "iterations": it, "max_true_relres": max(rr), "status": st, "zero_pivots": zp,
                     "ms_per_iteration": (t2 - t1) * 1e3 / max(1, it)}
    return out


def run_serve(args):
    from paper_1706_02205_gb300 import serve
    args.serve_fracs = (0.5, 0.8, 0.95)
    return serve.bench(args)


# ------------------------------------------------------- oracle (CPU) arm

def oracle_step(n_side, args):
    """One pass of the path in the FP64 oracle on a jittered grid n_side^2."""
    import oracle
    x = inputs.jittered_grid(n_side, seed=inputs.seed_for(2, 50))
    N = x.shape[0]
    b = inputs.rhs(N, args.nrhs, seed=inputs.seed_for(2, 51))
    t0 = time.perf_counter()
    perm, l, rp, col = oracle.sortsparse(x, args.rho)
    xo = x[perm]
    kern = oracle.Kernel(args.nu, args.ell)
    val, zc = oracle.ichol(xo, rp, col, kern)
    dg = oracle.solve_diag(xo, rp, val, kern)
    for r in range(args.nrhs):
        y = oracle.solve_lower(rp, col, val, dg, b[r][perm])
        oracle.solve_upper(rp, col, val, dg, y)
    dt = time.perf_counter() - t0
    return int(rp[-1]), dt, N


def cpu_baseline(args):
    side = args.cpu_baseline_side
    nnz, dt, N = oracle_step(side, args)
    return {"value": nnz / dt, "unit": "nnz(L)/s", "cores": 1, "kind": "oracle",
            "sample": f"jittered grid {side}x{side} (N={N}, {N / (args.n_side ** 2):.3g} of the workload's points), "
                      f"same kernel/rho/{args.nrhs} rhs; one full step (order+pattern+factor+solve) "
                      f"single-threaded FP64 C, {dt:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    for _ in range(args.warmup):
        oracle_step(args.cpu_side, args)
    tot, nnz_tot, N = 0.0, 0, 0
    for _ in range(args.steps):
        nnz, dt, N = oracle_step(args.cpu_side, args)
        tot += dt
        nnz_tot += nnz
    v = nnz_tot / tot
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "nnz(L)/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"jittered grid {args.cpu_side}x{args.cpu_side} (N={N}) sample of the "
                                   f"{args.n_side}x{args.n_side} workload, Matern-{args.nu} l={args.ell}, "
                                   f"rho={args.rho}, {args.nrhs} rhs"},
            "cpu_baseline": {"value": v, "unit": "nnz(L)/s", "cores": 1, "kind": "oracle",
                             "sample": f"jittered grid {args.cpu_side}^2 per step"},
            "e2e": {"value": v, "unit": "nnz(L)/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-side", type=int, default=1024)
    ap.add_argument("--nu", type=float, default=0.5)
    ap.add_argument("--other-nu", type=float, nargs="*", default=[1.5])
    ap.add_argument("--ell", type=float, default=0.1)
    ap.add_argument("--rho", type=float, default=3.0)
    ap.add_argument("--nrhs", type=int, default=16)
    ap.add_argument("--cpu-side", type=int, default=320, help="reference arm: jittered grid side of each step")
    ap.add_argument("--cpu-baseline-side", type=int, default=512,
                    help="cpu_baseline: jittered grid side of the bounded sample (1024 = the whole workload)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--traffic", type=float, default=None, help="ncu DRAM bytes per factor launch, if measured")
    ap.add_argument("--family", default="matern", choices=["matern", "cauchy"],
                    help="covariance family of the factor-only and tasks workloads")
    ap.add_argument("--alpha", type=float, default=1.0, help="Cauchy alpha")
    ap.add_argument("--shift", type=float, default=100.0, help="pde workload: zeroth-order term of the operator")
    ap.add_argument("--beta", type=float, default=0.2, help="Cauchy beta")
    ap.add_argument("--workload", default="grid2d",
                    choices=["grid2d", "cube3d", "factor", "batch", "serve", "refine", "tasks", "pde",
                             "supernodal"],
                    help="grid2d: the headline step (default); cube3d: 3-D factor + PCA; factor: factor-only "
                         "probe; batch: many sets in one launch; serve: request stream")
    ap.add_argument("--n3", type=int, default=2**18)
    ap.add_argument("--n-sets", type=int, default=256)
    ap.add_argument("--geom", default="grid2d", choices=["grid2d", "cube3d"], help="factor-only probe geometry")
    ap.add_argument("--rpt", type=int, nargs="*", default=[0], help="factor-only: rows per task (0 = default)")
    ap.add_argument("--lanes", type=int, nargs="*", default=[0], help="factor-only: lanes per row (0 = auto)")
    ap.add_argument("--unroll", type=int, nargs="*", default=[0], help="factor-only: staging depth (0 = 8)")
    ap.add_argument("--adaptive", type=int, nargs="*", default=[0], help="factor-only: adaptive chunks")
    ap.add_argument("--stage", type=int, nargs="*", default=[0],
                    help="factor-only: stage-buffer bytes (0 = automatic, -1 = register form)")
    ap.add_argument("--warps", type=int, nargs="*", default=[0], help="factor-only: warps per CTA (0 = default)")
    ap.add_argument("--n-req", type=int, default=40)
    ap.add_argument("--refine-side", type=int, default=256,
                    help="grid side of the refined-solve leg (0: leave it out)")
    ap.add_argument("--other-rho", type=float, nargs="*", default=[2.0, 5.0],
                    help="patterns of the configuration also factored (kernels timed)")
    ap.add_argument("--no-serve-leg", dest="serve_leg", action="store_false")
    ap.add_argument("--no-supernodal-leg", dest="supernodal_leg", action="store_false")
    ap.add_argument("--no-config-legs", dest="config_legs", action="store_false",
                    help="leave out the 3-D configuration and the batched launch from the default line")
    ap.add_argument("--e-reps", type=int, default=50, help="repetitions of the sampled error estimator")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--serve-n-max", type=int, default=1_000_000)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    args = ap.parse_args()

    from paper_1706_02205_gb300 import replicas
    rank, world = replicas.rank_world()
    if world > 1 and args.impl == "ours":
        replicas.init("nccl")
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    elif args.workload == "factor":
        line = run_factor_only(args)
    elif args.workload == "cube3d":
        line = run_cube3d(args)
    elif args.workload == "batch":
        line = run_batch(args)
    elif args.workload == "serve":
        line = run_serve(args)
    elif args.workload == "tasks":
        line = run_tasks(args)
    elif args.workload == "pde":
        line = run_pde(args)
    elif args.workload == "supernodal":
        line = run_supernodal(args)
    elif args.workload == "refine":
        line = run_refine(args)
    else:
        line = run_ours(args, rank, world)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
