#!/usr/bin/env python3
"""Benchmark: f(A) b time-to-1e-8 relative error, double-pass vs single-pass
multi-shift BiCGstab(l), and hop-kernel (stencil) GB/s against the HBM roofline.

Default workload: 16^3 x 32 Wilson-Dirac lattice, U = exp(i 0.4 H) (seeded),
mu = 0.1, m = -1.8, antiperiodic time, l = 2, Neuberger PFE with 20 poles,
A scaled by a power-iteration estimate of its largest eigenvalue; synthetic
stand-in for the paper's quenched gauge ensembles.

One step = one solve y = f(A) b by the pseudo-double-pass form (pass 1
stores the seed-vector occurrences, the sweep weights them, one gather forms
y; no shift vectors) in mixed precision (FP64 head until every live shift
residual is below switch_resid |b|, then FP32 bulk with FP64 scalars), with b
resident on the device and L2 flushed before each step.  value = mean ms per
solve (lower is better).  The same line reports the double-pass (pass 2
regenerates the vectors) mixed/FP64/FP32 and the single-pass FP64 solves,
each at the loosest tolerance whose result meets 1e-8 relative error against
a tol = 1e-12 FP64 solve.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl fapath|reference]

With torchrun (N > 1) each rank solves its own replica of the workload (the
solves are independent; no collective on the data path): scaling "weak".
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

import numpy as np  # noqa: E402

METRIC = "f(A)b time-to-1e-8 rel err (double vs single pass); stencil GB/s vs HBM peak"
TARGET = 1e-8
TOLS = (1e-8, 3e-9, 1e-9, 3e-10, 1e-10, 3e-11, 1e-11)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="fapath", choices=["fapath", "reference"])
    p.add_argument("--workload", default="wilson_16x16x16x32")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-large", action="store_true", help="skip the 32^3 x 64 variant of the default line")
    p.add_argument("--no-batched", action="store_true", help="skip the 72-system batched variant of the default line")
    p.add_argument("--switch-resid", type=float, default=-1.0,
                   help="head/tail switch threshold of the mixed forms; < 0: 0.08/l^2 (on 16^3 x 32, "
                        "l = 2 the fastest threshold whose error floor stays below half of 1e-8); "
                        "0: the library default min(0.04/l^2, 0.4/l^6)")
    p.add_argument("--quick", action="store_true",
                   help="headline solve only at tol 1e-9 (no comparisons, e2e or CPU baseline)")
    p.add_argument("--hop-only", action="store_true",
                   help="time D_w sweeps alone (FP32 and FP64) on --dims, for profiling")
    p.add_argument("--dims", type=int, nargs=4, default=None)
    p.add_argument("--ns-list", type=int, nargs="+", default=[2, 4, 8, 16, 32, 64],
                   help="numbers of poles of the --ns-sweep")
    p.add_argument("--ells", type=int, nargs="+", default=[1, 2, 4, 8], help="l values of the --ns-sweep")
    p.add_argument("--reps", type=int, default=20)
    p.add_argument("--head", default="mixed_df", choices=["mixed_df", "mixed"],
                   help="precision of the head of the headline solve: double-float or FP64")
    p.add_argument("--store-gb", type=float, default=0.0,
                   help="pseudo-double-pass store budget (0: the library default)")
    p.add_argument("--no-gram-epilogue", action="store_true",
                   help="FP32 stretches with the MR Gram matrix in a kernel of its own (by default the last "
                        "D_w sweep of each outer iteration forms it in its epilogue)")
    p.add_argument("--ns-sweep", action="store_true",
                   help="runtime against the number of poles at a fixed number of BiCG steps "
                        "(M l = 64) for the single-pass, double-pass and pseudo-double-pass forms")
    return p.parse_args()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist, device):
    """The replicas solve independent systems: the job's time per step is the
    slowest rank's (barrier + MAX all-reduce of one scalar, no data exchange)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ------------------------------------------------------------------ oracle baseline (CPU)
def oracle_sample(w, c, outer=1):
    """Time `outer` outer iterations of the oracle's seed recurrence (the work
    of one outer iteration of either pass of the oracle's double-pass form)."""
    from oracle import dirac, msbicgstab as ms
    op = dirac.Operator(w["U"], w["mass"], w["mu"], c, w["t_bc"])
    t0, c0 = time.perf_counter(), time.process_time()
    ms.seed_recurrence(op.A, w["b"], w["ell"], outer)
    t, cpu = time.perf_counter() - t0, time.process_time() - c0
    # threads actually used: process CPU time over wall time (numpy's stacked
    # 3x3 products and elementwise loops run on one thread)
    oracle_sample.threads = max(1, round(cpu / t))
    return t


def golden_outer_iters(name, tol=1e-9):
    """The oracle's own outer-iteration count for the workload, stored by
    tests/golden/make_golden.py, from the stored run whose tolerance is nearest
    to `tol` on a log scale (returns the count and that tolerance)."""
    import glob
    best = None
    for path in glob.glob(os.path.join(ROOT, "tests", "golden", f"{name}*.json")):
        with open(path) as f:
            g = json.load(f)
        if g.get("workload") != name or "outer_iters" not in g:
            continue
        d = abs(np.log10(g["tol"]) - np.log10(tol))
        if best is None or d < best[0]:
            best = (d, g["outer_iters"], g["tol"])
    return (best[1], best[2]) if best else (None, None)


def oracle_site_samples(name):
    """y* of the workload at sampled sites (all 12 spin-colour components of 48
    sites in every time slice), stored by tests/golden/make_golden.py --sites
    from the FP64 oracle at tol 1e-12; None when no such file exists."""
    path = os.path.join(ROOT, "tests", "golden", f"{name}_sites.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        g = json.load(f)
    idx = np.asarray(g["site_index_tzyx"])
    want = np.asarray(g["y_re"]) + 1j * np.asarray(g["y_im"])
    return {"index": idx, "y": want, "tol": g["tol"], "entries": int(want.size),
            "source": f"tests/golden/{name}_sites.json (FP64 oracle, tol {g['tol']:g})"}


def err_vs_oracle(y, samples):
    """Relative 2-norm of y - y* over the stored oracle samples, and max |dy| / max |y*|."""
    if samples is None:
        return None
    idx = samples["index"]
    yy = np.asarray(y)[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]].reshape(len(idx), 12)
    d = yy - samples["y"]
    return {"rel_2norm": float(np.linalg.norm(d) / np.linalg.norm(samples["y"])),
            "max_abs_over_max": float(np.abs(d).max() / np.abs(samples["y"]).max()),
            "entries": samples["entries"], "reference": samples["source"]}


def cpu_model():
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def oracle_anchor(name="wilson_4x4x4x8", tol=1e-10):
    """One whole double-pass solve of the FP64 oracle, timed end to end (no
    extrapolation): the power-iteration scale c, then f(A) b."""
    import inputs
    from oracle import dirac, msbicgstab as ms, poles, scale
    w = inputs.make_workload(name)
    t0 = time.perf_counter()
    op = dirac.Operator(w["U"], w["mass"], w["mu"], 1.0, w["t_bc"])
    c = scale.power_scale(op.A, w["v0"], 100)
    op = dirac.Operator(w["U"], w["mass"], w["mu"], c, w["t_bc"])
    om, sg = poles.neuberger_poles(w["ns"])
    st = ms.Stats()
    t1 = time.perf_counter()
    ms.multishift_double(op.A, w["b"], sg, om, w["ell"], tol, stats=st)
    t2 = time.perf_counter()
    return {"workload": name, "tol": tol, "solve_ms": (t2 - t1) * 1e3, "scale_ms": (t1 - t0) * 1e3,
            "outer_iters": st.n_outer, "extrapolated": False,
            "what": "one whole FP64 oracle double-pass solve, timed end to end"}


def cpu_baseline(w, c, outer_ref, outer=2, ref_tol=None):
    t = oracle_sample(w, c, outer)
    per_solve_ms = t / outer * 2 * outer_ref * 1e3
    at = f" (the oracle's own count at tol {ref_tol:g})" if ref_tol else ""
    return {"value": per_solve_ms, "unit": "ms", "cores": oracle_sample.threads, "kind": "oracle",
            "extrapolated": True, "per_outer_iteration_ms": t / outer * 1e3,
            "outer_iterations_scaled_to": 2 * outer_ref, "anchor": oracle_anchor(),
            "sample": f"{outer} outer iterations of the FP64 numpy oracle's BiCGstab({w['ell']}) "
                      f"recurrence on {'x'.join(map(str, w['dims']))} ({t:.1f} s), scaled by "
                      f"2 x {outer_ref} outer iterations{at} (pass 1 + pass 2 of the double-pass form); "
                      f"numpy, {oracle_sample.threads} thread(s) by CPU time / wall time, of "
                      f"{os.cpu_count()} host cores ({cpu_model()})"}


def run_reference(args, ws, rank):
    """Reference arm: the FP64 CPU oracle as it stands, rank 0 only."""
    if rank != 0:
        return
    import inputs
    from oracle import dirac, scale
    w = inputs.make_workload(args.workload)
    op = dirac.Operator(w["U"], w["mass"], w["mu"], 1.0, w["t_bc"])
    c = scale.power_scale(op.A, w["v0"], 100)
    outer_ref, ref_tol = golden_outer_iters(args.workload)
    if outer_ref is None:
        outer_ref, ref_tol = 100, None
    for _ in range(args.warmup):
        oracle_sample(w, c, 1)
    ts = [oracle_sample(w, c, 1) for _ in range(args.steps)]
    per_solve = statistics.mean(ts) * 2 * outer_ref * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": per_solve, "unit": "ms", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_solve, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args.workload, w),
        "cpu_baseline": {"value": per_solve, "unit": "ms", "cores": oracle_sample.threads, "kind": "oracle",
                         "extrapolated": True, "per_outer_iteration_ms": statistics.mean(ts) * 1e3,
                         "outer_iterations_scaled_to": 2 * outer_ref, "anchor": oracle_anchor(),
                         "sample": (f"each step: 1 outer iteration of the FP64 numpy oracle's "
                                    f"BiCGstab({w['ell']}) recurrence, scaled by 2 x {outer_ref} outer "
                                    f"iterations (both passes of the oracle's double-pass solve; "
                                    + (f"the oracle's own iteration count at tol {ref_tol}); " if ref_tol
                                       else "no stored oracle count for this workload, 100 assumed); ")
                                    + f"{oracle_sample.threads} thread(s) of {os.cpu_count()} host cores "
                                    f"({cpu_model()})")},
        "e2e": {"value": per_solve, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(name, w):
    return {"workload": name, "lattice": "x".join(map(str, w["dims"])), "ell": w["ell"], "ns": w["ns"],
            "mu": w["mu"], "mass": w["mass"], "eps": w["eps"], "poles": "neuberger",
            "target_rel_err": TARGET, "l2": "flushed before every timed step (512 MB write)"}


# ------------------------------------------------------------------ hop kernels alone
def run_hop_only(args):
    """D_w sweeps on the workload's gauge recipe at --dims: CUDA-event mean per
    launch and GB/s on the algorithmic bytes (FP32: 384 B/site, FP64: 960 B/site)."""
    import torch
    import inputs
    import paper_1010_2592_gb300 as fa
    w = inputs.make_workload(args.workload, tuple(args.dims) if args.dims else None)
    dims = w["dims"]
    V = int(np.prod(dims))
    ctx = fa.Context(dims)
    ctx.set_gauge(torch.from_numpy(w["U"]).cuda())
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], 1.0)
    x = torch.from_numpy(w["b"]).cuda()
    out = {}
    for prec, bytes_site in (("f32", 384.0), ("f64", 960.0), ("df", 960.0)):
        ctx.hop_timing_reset()
        y = ctx.empty_spinor()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(args.reps):
            ctx.apply_dw(x, precision=prec, out=y)
        e.record()
        torch.cuda.synchronize()
        ms_call = s.elapsed_time(e) / args.reps
        out[prec] = {"ms_per_apply_dw_call_incl_pack": ms_call}
    # the hop kernel alone: time a solve-free loop of hop launches via the solver's instrumentation
    solver_prec = {"f32": "f32", "f64": "f64", "df": "mixed_df"}
    for prec in ("f32", "f64", "df"):
        ctx.hop_timing_reset()
        ctx.set_poles(*fa.neuberger_poles(4))
        ctx.apply_f(x, ell=1, tol=1e-30, max_outer=max(1, args.reps // 4), mode="double",
                    precision=solver_prec[prec], switch_resid=1e-300, hop_timing=True, check=False)
        ms, n = ctx.hop_timing(prec)
        bsite = 384.0 if prec == "f32" else 960.0
        out[prec].update(hop_mean_ms=ms, hop_launches=n, hop_gbs=bsite * V / (ms * 1e-3) / 1e9 if ms else None)
    print(json.dumps({"mode": "hop-only", "dims": list(dims), "sites": V, **out}), flush=True)


# ------------------------------------------------------------------ batched workload
def run_ns_sweep(args):
    """Runtime against N_s at a fixed number of BiCG steps (the setting of the
    paper's Fig. 2, Sec. 3, which uses M l = 256 on 4^3 x 8): every solve runs
    exactly 64 / l outer iterations (the fixed-cost flag; the seed needs about
    100 BiCG steps to reach tol 1e-10 on this operator, so none stops early),
    FP64, on the workload's lattice (or --dims).  Shifts freeze when they
    converge, as in any solve (unfrozen, the zeta of the large shifts overflow
    FP64 within a few hundred steps).  One JSON line per (form, l): ms per solve
    for each N_s."""
    import torch
    import inputs
    import paper_1010_2592_gb300 as fa
    w = inputs.make_workload(args.workload, args.dims)
    dims = w["dims"]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = fa.Context(dims, stream)
    ctx.set_gauge(torch.from_numpy(w["U"]).cuda())
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], 1.0)
    c = ctx.estimate_scale(torch.from_numpy(w["v0"]).cuda(), 100)
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], c)
    b = torch.from_numpy(w["b"]).cuda()
    ns_list = tuple(args.ns_list)
    V = int(np.prod(dims))
    free, _ = torch.cuda.mem_get_info()
    for ell in args.ells:
        M = 64 // ell
        for form in ("single", "double", "pseudo"):
            row = {"mode": "ns_sweep", "lattice": "x".join(map(str, dims)), "ell": ell, "outer_iters": M,
                   "form": form, "precision": "f64", "ms": {}}
            for ns in ns_list:
                # the single-pass form holds N_s (l + 2) FP64 shift spinors
                if form == "single" and ns * (ell + 2) * 192.0 * V > 0.6 * free:
                    row.setdefault("skipped_ns", []).append(ns)
                    continue
                ctx.set_poles(*fa.neuberger_poles(ns))
                kw = dict(ell=ell, tol=1e-10, max_outer=M, mode=form, precision="f64", fixed_iters=True,
                          store_gb=0.5 * free / 1e9 if form == "pseudo" else 0.0)
                ctx.apply_f(b, **kw)
                times = []
                for _ in range(max(1, args.steps)):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    r = ctx.apply_f(b, **kw)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                row["ms"][str(ns)] = statistics.median(times)
                row.setdefault("outer_iters_run", {})[str(ns)] = r.stats["outer_iters"]
                row.setdefault("status", r.stats["status"])
            print(json.dumps(row), flush=True)
    ctx.close()


def batched_measure(steps, warmup, ells=None, one_at_a_time=True, name="wilson_batched_72", store_gb=0.0,
                    with_head=True):
    """72 systems: 12 spin-colour point sources on each of 6 lattices of three
    shapes (2 x 8^4, 2 x 12^3 x 24, 2 x 16^3 x 32), mu_k ~ U[0, 0.2], 16 Neuberger
    poles, FP32 bulk, pseudo-double-pass.  One step = one fa_apply_f_batched
    call over all 72 systems; compared with the same 72 solves one at a time,
    and the first source of every lattice against an FP64 solve."""
    import torch
    import inputs
    import paper_1010_2592_gb300 as fa
    w = inputs.make_batched_workload(name)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctxs, srcs, owners = [], [], []
    om, sg = fa.neuberger_poles(w["ns"])
    for lat in w["lattice_systems"]:
        owner = fa.Context(lat["dims"], stream)
        owner.set_gauge(torch.from_numpy(lat["U"]).cuda())
        owner.set_params(w["mass"], lat["mu"], w["t_bc"], 1.0)
        c = owner.estimate_scale(torch.from_numpy(lat["v0"]).cuda(), 100)
        for k, src in enumerate(lat["sources"]):
            ctx = owner if k == 0 else fa.Context(lat["dims"], stream)
            if k > 0:
                ctx.share_gauge(owner)
            ctx.set_params(w["mass"], lat["mu"], w["t_bc"], c)
            ctx.set_poles(om, sg)
            ctxs.append(ctx)
            srcs.append(torch.from_numpy(src).cuda())
        owners.append(owner)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, total = torch.cuda.mem_get_info()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    out = {"workload": name, "systems": len(ctxs), "ns": w["ns"],
           "lattices": ["x".join(map(str, l["dims"])) for l in w["lattice_systems"]],
           "mu": [round(l["mu"], 4) for l in w["lattice_systems"]], "form": "pseudo",
           "launches": "one launch per kernel for all 72 systems (work tables); FP32 sweeps by lattice group",
           "l2": "flushed before every timed step (512 MB write)",
           "free_gb_at_start": free / 1e9, "device_gb": total / 1e9}
    tune = fa.autotune_batched(ctxs, reps=5)   # multi-RHS sweep shape for this batch (untimed)
    out["mrhs_shape"] = {"rhs_per_block": tune["rhs_per_block"], "min_blocks": tune["min_blocks"]}
    # FP32 bulk at l = 2 and l = 4; at l = 4 the FP32-only form stays above 1e-6
    # (power-basis cancellation), so the same batch also runs with a double-float head
    # (the head switches at 0.04/l^2 = 0.0025: the batch's bound is 1e-6, which
    # this meets with orders of magnitude to spare, for fewer head iterations)
    runs = [(ell, "f32") for ell in (ells or w["ell"])] + ([(4, "mixed_df")] if with_head else [])
    for ell, precision in runs:
        kw = dict(ell=ell, tol=w["tol"], max_outer=4000, mode="pseudo", precision=precision,
                  store_gb=store_gb if store_gb > 0 else 0.4 * free / 1e9, graph=True,
                  switch_resid=0.04 / ell ** 2 if precision != "f32" else 0.0)
        ys, st = fa.apply_f_batched(ctxs, srcs, **kw)          # warm-up (also instantiates graphs)
        for _ in range(max(0, warmup - 1)):
            fa.apply_f_batched(ctxs, srcs, **kw)
        times = []
        torch.cuda.nvtx.range_push(f"batched_l{ell}_{precision}")
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ys, st = fa.apply_f_batched(ctxs, srcs, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        torch.cuda.nvtx.range_pop()
        row = {"ms_batched": statistics.mean(times), "systems_per_s": len(ctxs) / (statistics.mean(times) * 1e-3),
               "outer_iters_max": max(x["outer_iters"] for x in st),
               "outer_iters_min": min(x["outer_iters"] for x in st),
               "stored_outer": st[0]["stored_outer"], "store_gb": kw["store_gb"]}
        if one_at_a_time:
            # the same 72 solves, one at a time, each with its share of the store budget
            kw1 = dict(kw, store_gb=kw["store_gb"] / len(ctxs))
            for ctx, b in zip(ctxs[:3], srcs[:3]):
                ctx.apply_f(b, **kw1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for ctx, b in zip(ctxs, srcs):
                ctx.apply_f(b, **kw1)
            torch.cuda.synchronize()
            one = (time.perf_counter() - t0) * 1e3
            row.update(ms_one_at_a_time=one, speedup=one / statistics.mean(times))
        # accuracy of the FP32 bulk against an FP64 solve, first source of every lattice
        errs = []
        for k in range(0, len(ctxs), 12):
            r64 = ctxs[k].apply_f(srcs[k], ell=ell, tol=1e-12, max_outer=4000, mode="double", precision="f64")
            errs.append(float((torch.linalg.vector_norm(ys[k] - r64.y) / torch.linalg.vector_norm(r64.y)).item()))
        row["rel_err_vs_f64_per_lattice"] = errs
        row["precision"] = precision
        out[f"ell{ell}" + ("" if precision == "f32" else "_" + precision)] = row
    for c_ in ctxs:
        c_.close()
    return out


def run_batched(args):
    """--workload wilson_batched_72: the batch alone (with --quick: l 2, FP32 only,
    without the one-at-a-time comparison)."""
    out = batched_measure(args.steps, args.warmup, ells=(2,) if args.quick else None,
                          one_at_a_time=not args.quick, store_gb=args.store_gb, with_head=not args.quick)
    print(json.dumps(dict(mode="batched", **out)), flush=True)


def large_measure(steps, warmup, name="wilson_32x32x32x64"):
    """The 32^3 x 64 workload (l 4, 32 poles): pseudo-double-pass with a
    double-float head and FP32 tail, at the loosest tolerance of TOLS whose
    result meets 1e-8 against an FP64 double-pass solve at tol 1e-12 (the FP64
    oracle would take hours here); L2 flushed before every timed step; the FP32
    sweep's event-timed bandwidth inside the instrumented repeat.  Head/tail
    switch at 0.04/l^2 |b| (a scan of 1e-4 ... 2.5e-3 on this workload: the error
    stays at 1.4e-9 - 3.5e-9 at tol 1e-9 and 7.5e-9 - 9.9e-9 at tol 3e-9 while the
    head shrinks from 12 to 6 outer iterations)."""
    import torch
    import inputs
    import paper_1010_2592_gb300 as fa
    w = inputs.make_workload(name)
    dims, ell = w["dims"], w["ell"]
    V = int(np.prod(dims))
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = fa.Context(dims, stream)
    ctx.set_gauge(torch.from_numpy(w["U"]).cuda())
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], 1.0)
    c = ctx.estimate_scale(torch.from_numpy(w["v0"]).cuda(), 100)
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], c)
    ctx.set_poles(*fa.neuberger_poles(w["ns"]))
    b = torch.from_numpy(w["b"]).cuda()
    ns = w["ns"]
    del w
    torch.cuda.empty_cache()
    free, total = torch.cuda.mem_get_info()
    ref = ctx.apply_f(b, ell=ell, tol=1e-12, max_outer=4000, mode="double", precision="f64")
    yref, yn = ref.y, torch.linalg.vector_norm(ref.y).item()
    kw = dict(ell=ell, max_outer=4000, mode="pseudo", precision="mixed_df", switch_resid=0.04 / ell ** 2,
              graph=True, store_gb=0.8 * free / 1e9)
    pick = None
    for tol in TOLS:
        r = ctx.apply_f(b, tol=tol, check=False, **kw)
        e = (torch.linalg.vector_norm(r.y - yref) / yn).item() if r.stats["status"] == 0 else float("inf")
        pick = (tol, e, r.stats)
        if e <= TARGET:
            break
    tol, e, st = pick
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        ctx.apply_f(b, tol=tol, **kw)
    times = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.apply_f(b, tol=tol, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ctx.hop_timing_reset()
    ctx.apply_f(b, tol=tol, hop_timing=True, **dict(kw, graph=False))
    hop_ms, hop_n = ctx.hop_timing("f32", dot=False)
    peak, _ = measured_hbm_peak()
    gbs = 384.0 * V / (hop_ms * 1e-3) / 1e9 if hop_ms else None
    out = {"workload": name, "lattice": "x".join(map(str, dims)), "ell": ell, "ns": ns,
           "ms": statistics.mean(times), "tol": tol, "rel_err_vs_f64": e, "meets_1e-8": e <= TARGET,
           "reference": "the library's FP64 double-pass solve at tol 1e-12", "outer_iters": st["outer_iters"],
           "switch_outer": st["switch_outer"], "switch_resid": kw["switch_resid"], "stored_outer": st["stored_outer"],
           "free_gb_at_start": free / 1e9, "store_gb": kw["store_gb"], "device_gb": total / 1e9,
           "hop_f32_plain": {"mean_launch_ms": hop_ms, "launches": hop_n, "gbs": gbs,
                             "frac_of_measured_hbm": gbs / peak if gbs else None,
                             "bytes_per_launch": 384.0 * V},
           "l2": "flushed before every timed step (512 MB write)"}
    ctx.close()
    return out


def trace_timeline(ctx, run, stats, V):
    """One more graph-replayed solve with the kernel timeline tracer on
    (fa_trace_start / fa_trace_stop): every block's entry and exit time, so the
    launches are timed as they run in the replayed graphs, with nothing between
    them.  Pass-1 outer iteration m is the run of launches that ends with its
    k_mr; the first `switch_outer` are the double-float head, the rest up to
    `outer_iters` the FP32 tail (iterations enqueued past convergence return at
    once and are left out).  Returns the per-kernel spans of the FP32 tail, the
    time per outer iteration, and the plain FP32 sweep's mean span."""
    import paper_1010_2592_gb300 as fa
    fa.trace_start(1 << 22)
    try:
        run()
    finally:
        rec, dropped = fa.trace_stop(1 << 22)
    launches = fa.trace_launches(rec)
    M, sw = stats["outer_iters"], max(0, stats["switch_outer"])
    iters, cur = [], []
    for L in launches:
        cur.append(L)
        if L["name"].startswith("k_mr<") and len(iters) < M:
            iters.append(cur)
            cur = []
    if len(iters) < M:
        return {"error": f"{len(iters)} outer iterations traced of {M}", "dropped": dropped}

    def summary(lo, hi):
        if hi <= lo:
            return None
        per = {}
        for it in iters[lo:hi]:
            for L in it:
                d = per.setdefault(L["name"], [0, 0.0, 0.0])
                d[0] += 1
                d[1] += (L["end_ns"] - L["start_ns"]) / 1e3
                d[2] += L["tail_ns"] / 1e3
        n = hi - lo
        # iteration time: first launch of iteration k to first launch of k + 1
        spans = [iters[k + 1][0]["start_ns"] - iters[k][0]["start_ns"] for k in range(lo, min(hi, M - 1))]
        busy = sum(L["end_ns"] - L["start_ns"] for it in iters[lo:hi] for L in it) / n / 1e3
        per_it = sum(spans) / len(spans) / 1e3 if spans else None
        return {"outer_iterations": n, "us_per_outer_iteration": per_it, "kernel_us_per_outer_iteration": busy,
                "gaps_us_per_outer_iteration": (per_it - busy) if per_it else None,
                "kernels": {k: {"launches_per_iteration": v[0] / n, "mean_span_us": v[1] / v[0],
                                "mean_last_block_tail_us": v[2] / v[0]} for k, v in per.items()}}
    tail = iters[sw:M]
    plain = [L for it in tail for L in it if L["name"] == "k_hop1<f32>"]
    mean_ms = sum(L["end_ns"] - L["start_ns"] for L in plain) / len(plain) / 1e6 if plain else None
    # every launch of the solve (pass 1 to the end of pass 2) up to the last
    # outer iteration that did work, per kernel: launches, summed span
    last = iters[M - 1][-1]["end_ns"]
    per_kernel = {}
    for L in launches:
        if L["end_ns"] <= last or not L["name"].startswith(("k_update", "k_hop", "k_mr", "k_gram")):
            d = per_kernel.setdefault(L["name"], [0, 0])
            d[0] += 1
            d[1] += L["end_ns"] - L["start_ns"]
    solve_ns = launches[-1]["end_ns"] - launches[0]["start_ns"]
    return {"fp32_tail": summary(sw, M), "double_float_head": summary(0, sw), "dropped": dropped,
            "launches_traced": len(launches), "hop_f32_plain_mean_ms": mean_ms, "hop_f32_plain_launches": len(plain),
            "pass1_us": (iters[M - 1][-1]["end_ns"] - iters[0][0]["start_ns"]) / 1e3,
            "traced_solve_us": solve_ns / 1e3,
            "per_kernel": {k: {"launches": v[0], "total_us": v[1] / 1e3, "mean_us": v[1] / v[0] / 1e3}
                           for k, v in sorted(per_kernel.items(), key=lambda kv: -kv[1][1])}}


def measured_hbm_peak():
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        with open(peaks_path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.hop_only:
        run_hop_only(args)
        return
    if args.ns_sweep:
        run_ns_sweep(args)
        return
    if args.workload == "wilson_batched_72":
        run_batched(args)
        return

    import torch
    import inputs
    import paper_1010_2592_gb300 as fa

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = inputs.make_workload(args.workload)
    dims, ell, ns = w["dims"], w["ell"], w["ns"]
    V = int(np.prod(dims))
    stream = torch.cuda.Stream()           # a capturable stream (graph replay)
    torch.cuda.set_stream(stream)
    ctx = fa.Context(dims, stream)
    ctx.set_gauge(torch.from_numpy(w["U"]).cuda())
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], 1.0)
    c = ctx.estimate_scale(torch.from_numpy(w["v0"]).cuda(), 100)
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], c)
    om, sg = fa.neuberger_poles(ns)
    ctx.set_poles(om, sg)
    tune = ctx.autotune(reps=20)        # FP32 sweep launch shape for this lattice (untimed)
    b = torch.from_numpy(w["b"]).cuda()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    # reference solutions for the error measurement (untimed): the library's own
    # FP64 solve at tol 1e-12 on the whole lattice, and the FP64 oracle's y* at
    # the sampled sites stored with the tests (when the workload has them)
    yref = ctx.apply_f(b, ell=ell, tol=1e-12, max_outer=4000, precision="f64").y
    yref_norm = torch.linalg.vector_norm(yref).item()
    samples = oracle_site_samples(args.workload)

    def err(y):
        return (torch.linalg.vector_norm(y - yref) / yref_norm).item()

    def err_o(y):
        return err_vs_oracle(y.cpu().numpy(), samples)

    if args.switch_resid < 0:
        args.switch_resid = 0.08 / ell ** 2
    variants = {
        "pseudo_mixed": dict(mode="pseudo", precision=args.head, switch_resid=args.switch_resid, graph=True,
                             store_gb=args.store_gb, gram_epilogue=not args.no_gram_epilogue),
        "pseudo_mixed_fp64head": dict(mode="pseudo", precision="mixed", switch_resid=args.switch_resid, graph=True,
                                      store_gb=args.store_gb),
        "double_mixed": dict(mode="double", precision="mixed", switch_resid=args.switch_resid),
        "double_f64": dict(mode="double", precision="f64"),
        "single_f64": dict(mode="single", precision="f64"),
        "double_f32": dict(mode="double", precision="f32"),
        # the 16^3 x 32 configuration's literal form: FP32 bulk with reliable updates
        # every 50 BiCG iterations (25 outer iterations of BiCGstab(2)), and the
        # headline with the same reliable updates
        "double_f32_reliable": dict(mode="double", precision="f32", reliable_every=25),
        "pseudo_mixed_reliable": dict(mode="pseudo", precision=args.head, switch_resid=args.switch_resid,
                                      graph=True, store_gb=args.store_gb, reliable_every=25),
    }
    chosen = {}
    if args.quick:
        variants = {"pseudo_mixed": variants["pseudo_mixed"]}
    if args.head == "mixed":
        variants.pop("pseudo_mixed_fp64head", None)
    for name, kw in variants.items():
        if args.quick:
            r = ctx.apply_f(b, ell=ell, tol=1e-9, max_outer=4000, **kw)
            chosen[name] = (1e-9, err(r.y), r.stats)
            continue
        pick = None
        for tol in TOLS:
            r = ctx.apply_f(b, ell=ell, tol=tol, max_outer=4000, check=False, **kw)
            e = err(r.y) if r.stats["status"] == 0 else float("inf")
            pick = (tol, e, r.stats)
            # the headline must also meet the target against the oracle's samples
            eo = err_o(r.y) if (name == "pseudo_mixed" and samples is not None) else None
            if e <= TARGET and (eo is None or eo["rel_2norm"] <= TARGET):
                break
        chosen[name] = pick

    def timed(name, steps, warmup, hop=False):
        kw = dict(variants[name])
        tol = chosen[name][0]
        for _ in range(warmup):
            ctx.apply_f(b, ell=ell, tol=tol, max_outer=4000, **kw)
        ms_list = []
        launches = 0
        last = None
        for _ in range(steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            n0 = ctx.launch_count()
            s.record(stream)
            last = ctx.apply_f(b, ell=ell, tol=tol, max_outer=4000, hop_timing=hop, **kw)
            e.record(stream)
            torch.cuda.synchronize()
            launches += ctx.launch_count() - n0
            ms_list.append(s.elapsed_time(e))
        return ms_list, launches, last

    # headline: pseudo-double-pass, mixed precision, each outer iteration replayed
    # from a captured CUDA graph
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    head_ms, head_launches, head_res = timed("pseudo_mixed", args.steps, args.warmup)
    torch.cuda.nvtx.range_pop()
    # the same steps once more with direct launches and CUDA events around every
    # hop-kernel launch (events cannot sit inside a replayed graph): the rooflines
    variants["pseudo_mixed_events"] = dict(variants["pseudo_mixed"], graph=False)
    chosen["pseudo_mixed_events"] = chosen["pseudo_mixed"]
    ctx.hop_timing_reset()
    inst_ms, _, _ = timed("pseudo_mixed_events", args.steps, 1, hop=True)
    clk = clocks.stop()
    torch.cuda.synchronize()
    ms_step = max_over_ranks(statistics.mean(head_ms), dist, "cuda")
    # the same solve once more, graph-replayed, with the kernel timeline tracer on
    try:
        kw_t = dict(variants["pseudo_mixed"])
        tol_t = chosen["pseudo_mixed"][0]
        timeline = trace_timeline(ctx, lambda: ctx.apply_f(b, ell=ell, tol=tol_t, max_outer=4000, **kw_t),
                                  head_res.stats, V)
    except Exception as ex:   # reported, never fatal to the bench line
        timeline = {"error": f"{type(ex).__name__}: {ex}"}
    hop32_ms, hop32_n = ctx.hop_timing("f32", dot=False)      # k_hop1<float, false>
    hop32d_ms, hop32d_n = ctx.hop_timing("f32", dot=True)     # k_hop1<float, true>
    hop64_ms, hop64_n = ctx.hop_timing("f64")
    hopdf_ms, hopdf_n = ctx.hop_timing("df", dot=False)       # k_hop1_rows<df, false>
    hopdfd_ms, hopdfd_n = ctx.hop_timing("df", dot=True)      # k_hop1_rows<df, true>
    hopg_ms, hopg_n = ctx.hop_timing("f32", dot="gram")       # k_hop_gram (Gram-matrix epilogue)

    # comparison variants (fewer steps)
    other = {}
    for name in ([] if args.quick else ["pseudo_mixed_fp64head", "double_mixed", "double_f64", "single_f64",
                                        "double_f32", "double_f32_reliable", "pseudo_mixed_reliable"]):
        if name not in variants:
            continue
        k = max(1, min(args.steps, 3))
        lst, _, res = timed(name, k, 1)
        tol, e, _ = chosen[name]
        other[name] = {"ms": statistics.mean(lst), "tol": tol, "rel_err": e,
                       "outer_iters": res.stats["outer_iters"], "meets_1e-8": e <= TARGET}
    tol_h, e_h, _ = chosen["pseudo_mixed"]
    if not args.quick:
        # the overlap operator of Sec. 1 with the headline's solve settings:
        # D_ov(mu) b = b + g5 sign(g5 D_w(mu)) b = b + sqrt(c) D_w f(A) b, error
        # against the same operator with an FP64 solve at tol 1e-12
        try:
            kw = dict(variants["pseudo_mixed"])
            ov_ref = ctx.apply_overlap(b, ell=ell, tol=1e-12, max_outer=4000, precision="f64").y
            for _ in range(2):
                ov = ctx.apply_overlap(b, ell=ell, tol=tol_h, max_outer=4000, **kw)
            lst = []
            for _ in range(max(1, min(args.steps, 3))):
                flush.zero_()
                s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                s_ev.record(stream)
                ov = ctx.apply_overlap(b, ell=ell, tol=tol_h, max_outer=4000, **kw)
                e_ev.record(stream)
                torch.cuda.synchronize()
                lst.append(s_ev.elapsed_time(e_ev))
            e_ov = (torch.linalg.vector_norm(ov.y - ov_ref) / torch.linalg.vector_norm(ov_ref)).item()
            other["overlap_pseudo_mixed"] = {
                "ms": statistics.mean(lst), "tol": tol_h, "rel_err_vs_f64_overlap": e_ov,
                "outer_iters": ov.stats["outer_iters"],
                "what": "D_ov(mu) b = b + g5 sign(g5 D_w(mu)) b through fa_apply_overlap (solve + one FP64 sweep)"}
        except Exception as ex:   # reported, never fatal to the bench line
            other["overlap_pseudo_mixed"] = {"error": f"{type(ex).__name__}: {ex}"}
    other["pseudo_mixed_events"] = {"ms": statistics.mean(inst_ms), "note": "direct launches, hop events on"}
    head_vs_oracle = err_o(head_res.y)
    other["pseudo_mixed"] = {"ms": ms_step, "tol": tol_h, "rel_err": e_h, "rel_err_vs_oracle": head_vs_oracle,
                             "rel_err_reference": "rel_err: the library's FP64 solve at tol 1e-12, whole lattice; "
                                                  "rel_err_vs_oracle: the FP64 oracle's y* at the stored samples",
                             "outer_iters": head_res.stats["outer_iters"],
                             "stored_outer": head_res.stats["stored_outer"],
                             "switch_outer": head_res.stats["switch_outer"], "meets_1e-8": e_h <= TARGET}

    if args.quick:
        print(json.dumps({"mode": "quick", "ms_per_solve": ms_step, "variant": other["pseudo_mixed"],
                          "rel_err_vs_oracle": head_vs_oracle,
                          "hop_f32_ms": hop32_ms, "hop_f32_dot_ms": hop32d_ms, "hop_f64_ms": hop64_ms,
                          "hop_df_ms": hopdf_ms, "hop_df_dot_ms": hopdfd_ms,
                          "hop_f32_gram_ms": ctx.hop_timing("f32", dot="gram")[0],
                          "gram_epilogue": not args.no_gram_epilogue,
                          "hop_f32_gbs": 384.0 * V / (hop32_ms * 1e-3) / 1e9 if hop32_ms else None,
                          "launches_per_solve": head_launches // max(1, args.steps), "clocks": clk,
                          "timeline": timeline}),
              flush=True)
        ctx.close()
        return

    # end to end through the host-buffer entry point: pinned b in, pinned y out
    b_pin = torch.from_numpy(w["b"]).pin_memory()
    y_pin = torch.empty_like(b_pin).pin_memory()
    kw = dict(variants["pseudo_mixed"])
    p = ctx.params(ell=ell, tol=tol_h, max_outer=4000, **kw)
    st = fa.SolverStats()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = ctx.lib.fa_apply_f_host(ctx.h, b_pin.data_ptr(), y_pin.data_ptr(), p, st)
        t1 = time.perf_counter()
        assert rc == 0, rc
        if i >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_err = float(np.linalg.norm(y_pin.numpy() - yref.cpu().numpy()) / yref_norm)
    e2e_err_o = err_vs_oracle(y_pin.numpy(), samples)

    # rooflines of the sweep kernels, each template instance on its own (the
    # plain sweep and the sweep that also forms <rt, out> and runs a seed step
    # are different kernels with different bytes); the one with the most device
    # time in the timed solves is reported as "roofline".
    #   FP32 sweep: HBM-bound, 96 B in + 96 B out + 4 x 48 B links = 384 B/site;
    #   with the inner product + 96 B of rt = 480 B/site.
    #   FP64 sweep: FP64-ALU-bound on GB300; 1704 FP64 flops/site counted from the
    #   kernel source (8 hops x (24 add projection + 12 mul + 60 fma link product
    #   + 48 add reconstruction) + 12 time-weight mul x 2 + 24 mul + 24 fma
    #   centre term; fma = 2 flops), against the nominal 1.25 TFLOP/s FP64.
    #   double-float sweep (row split, shared projection, compensated arithmetic):
    #   bound by FP32 issue; 11,650 thread instructions per site, the ncu
    #   instruction count of one plain 16^3 x 32 launch (smsp__inst_executed x 32
    #   / V), against 152 SMs x 128 FP32 lanes x 2.07 GHz = 40.3 T instructions/s.
    peak, peak_src = measured_hbm_peak()
    over = "the instrumented repeat of the timed steps (direct launches, CUDA events around each sweep launch)"

    def roof(kernel, bound, per_launch, ms, n, unit, pk, pk_src, what, scale):
        ach = per_launch / (ms * 1e-3) / scale if ms > 0 else None
        return {"kernel": kernel, "bound": bound, "measured_over": over, "achieved": ach, "peak": pk,
                "unit": unit, "frac": (ach / pk) if ach else None, "traffic": None, "peak_source": pk_src,
                what: per_launch, "mean_launch_ms": ms, "launches_timed": n, "total_ms": ms * n}

    roof32 = roof("k_hop1<float, false> (one D_w sweep, FP32 12-real links; 128-thread blocks, 7/SM)", "hbm",
                  384.0 * V, hop32_ms, hop32_n, "GB/s", peak, peak_src, "algorithmic_bytes_per_launch", 1e9)
    roof32d = roof("k_hop1<float, true> (D_w sweep + <rt, out> + seed step in the last block)", "hbm",
                   480.0 * V, hop32d_ms, hop32d_n, "GB/s", peak, peak_src, "algorithmic_bytes_per_launch", 1e9)
    roof64 = roof("k_hop1<double> (one D_w sweep, FP64; both instances)", "alu", 1704.0 * V, hop64_ms, hop64_n,
                  "TFLOP/s", 1.25, "nominal GB300 FP64 (no measured FP64 peak)", "algorithmic_flops_per_launch",
                  1e12)
    # the FP32 issue peak measured on this GPU by the library's probe (eight
    # independent FMA chains per thread, 2048 threads per SM); nominal
    # 152 SMs x 128 lanes x 2.07 GHz = 40.3 T/s if the probe fails
    try:
        rate, _ = fa.fp32_issue_rate(5)
        fp32_peak = rate / 1e12
        nom = "measured: fa_fp32_issue_rate (FP32 FMA probe, 8 independent chains per thread, 2048 threads/SM)"
    except Exception:
        fp32_peak = 40.3
        nom = "152 SMs x 128 FP32 lanes x 2.07 GHz (nominal; the probe failed)"
    roofdf = roof("k_hop1_rows<df, false> (one D_w sweep, double-float head, row split)", "alu", 11650.0 * V,
                  hopdf_ms, hopdf_n, "T FP32-instructions/s", fp32_peak, nom, "algorithmic_instructions_per_launch",
                  1e12)
    roofdfd = roof("k_hop1_rows<df, true> (sweep + <rt, out> + seed step; the sweep's instructions only)", "alu",
                   11650.0 * V, hopdfd_ms, hopdfd_n, "T FP32-instructions/s", fp32_peak, nom,
                   "algorithmic_instructions_per_launch", 1e12)
    achieved = roof32["achieved"]
    # DRAM traffic per launch from one ncu capture of the FP32 sweeps in the timed
    # solve on this lattice (dram__bytes_read.sum + dram__bytes_write.sum; means
    # over 2 + 2 launches); constants from that capture, applied only on its
    # lattice, null elsewhere and for the double-float sweeps (not re-captured)
    src = ("ncu capture (dram__bytes_read.sum + dram__bytes_write.sum per launch) of these kernels inside "
           "the 16^3x32 headline solve, profiles/hop_traffic_16x16x16x32.md; fixed constants, not "
           "re-measured by this run")
    for r_ in (roof32, roof32d, roof64, roofdf, roofdfd):
        r_["traffic_source"] = None
    if V == 16 * 16 * 16 * 32:
        roof32["traffic"] = 37.777e6 + 0.005e6
        roof32d["traffic"] = 50.423e6 + 0.183e6
        for r_ in (roof32, roof32d):
            r_["traffic_source"] = src
    roofg = roof(f"k_hop_gram<{ell}> (the outer iteration's last FP32 sweep with the Gram matrix in its epilogue)",
                 "hbm", (384.0 + 96.0 * ell) * V, hopg_ms, hopg_n, "GB/s", peak, peak_src,
                 "algorithmic_bytes_per_launch", 1e9)
    roofg["traffic_source"] = None
    # the plain FP32 sweep timed alone: the autotuner's chains of back-to-back
    # launches (each reads the previous one's output), replayed from a CUDA graph
    # as in the solve, between two CUDA events, against the burst copy peak
    alone_ms = min(tune["times_ms"]) if tune.get("times_ms") else None
    roof_alone = {"kernel": "k_hop1<float, false> timed alone (fa_autotune: a CUDA graph of 20 back-to-back "
                            "sweeps, best of three rounds, the faster shape)", "bound": "hbm", "achieved": 384.0 * V / (alone_ms * 1e-3) / 1e9
                  if alone_ms else None, "peak": peak, "unit": "GB/s", "peak_source": peak_src + " (burst copy)",
                  "mean_launch_ms": alone_ms, "algorithmic_bytes_per_launch": 384.0 * V, "traffic": None,
                  "traffic_source": None}
    roof_alone["frac"] = roof_alone["achieved"] / peak if roof_alone["achieved"] else None
    # the plain FP32 sweep inside the graph-replayed solve: mean span (first block
    # entry to last block exit) from the kernel timeline tracer, over the FP32
    # tail's launches of one traced repeat of the timed solve
    tr_ms = timeline.get("hop_f32_plain_mean_ms") if isinstance(timeline, dict) else None
    roof_graph = {"kernel": "k_hop1<float, false> inside the graph-replayed solve", "bound": "hbm",
                  "measured_over": "kernel spans (earliest block entry to latest block exit, %globaltimer, "
                                   "fa_trace_start/fa_trace_stop) of the FP32 tail of one graph-replayed repeat of "
                                   "the timed solve; no events or other work between the launches",
                  "achieved": 384.0 * V / (tr_ms * 1e-3) / 1e9 if tr_ms else None, "peak": peak, "unit": "GB/s",
                  "peak_source": peak_src, "mean_launch_ms": tr_ms,
                  "launches": timeline.get("hop_f32_plain_launches") if isinstance(timeline, dict) else None,
                  "algorithmic_bytes_per_launch": 384.0 * V, "traffic": roof32["traffic"],
                  "traffic_source": roof32["traffic_source"]}
    roof_graph["frac"] = roof_graph["achieved"] / peak if roof_graph["achieved"] else None
    roofs = [roof32, roof32d, roof64, roofdf, roofdfd, roofg]
    dominant_events = max(roofs, key=lambda r: r["total_ms"])
    # "roofline": the kernel with the most device time in the graph-replayed timed
    # solve, timed as it runs there (the tracer's span of each launch: earliest
    # block entry to latest block exit, no events between the launches); CUDA
    # events cannot sit inside a replayed graph, and around direct launches they
    # add the launch processing to every sweep (the events figure of the same
    # kernel is given beside it)
    per_k = timeline.get("per_kernel", {}) if isinstance(timeline, dict) else {}
    cand = {   # kernel name -> (bound, algorithmic work per launch, unit scale, peak, unit, peak source, events roofline)
        "k_hop1<f32>": ("hbm", 384.0 * V, 1e9, peak, "GB/s", peak_src, roof32),
        "k_hop1<f32, dot>": ("hbm", 480.0 * V, 1e9, peak, "GB/s", peak_src, roof32d),
        "k_hop_gram<f32>": ("hbm", (384.0 + 96.0 * ell) * V, 1e9, peak, "GB/s", peak_src, roofg),
        "k_hop1_rows<df>": ("alu", 11650.0 * V, 1e12, fp32_peak, "T FP32-instructions/s", nom, roofdf),
        "k_hop1_rows<df, dot>": ("alu", 11650.0 * V, 1e12, fp32_peak, "T FP32-instructions/s", nom, roofdfd),
    }
    in_graph = [k for k in per_k if k in cand]
    dominant = dominant_events
    if in_graph:
        kname = max(in_graph, key=lambda k: per_k[k]["total_us"])
        bound, work, scl, pk, unit, pk_src, ev = cand[kname]
        span_ms = per_k[kname]["mean_us"] * 1e-3
        ach = work / (span_ms * 1e-3) / scl
        top = next(iter(per_k))
        dominant = {
            "kernel": ev["kernel"], "trace_name": kname, "bound": bound,
            "measured_over": "kernel spans (earliest block entry to latest block exit, %globaltimer, "
                             "fa_trace_start/fa_trace_stop) of every launch in one graph-replayed repeat of the "
                             "timed solve; no events or other work between the launches",
            "achieved": ach, "peak": pk, "unit": unit, "frac": ach / pk, "peak_source": pk_src,
            ("algorithmic_bytes_per_launch" if bound == "hbm" else "algorithmic_instructions_per_launch"): work,
            "mean_launch_ms": span_ms, "launches": per_k[kname]["launches"],
            "total_ms": per_k[kname]["total_us"] * 1e-3,
            "share_of_traced_solve": per_k[kname]["total_us"] / timeline["traced_solve_us"],
            "kernel_with_most_device_time": top,
            "traffic": ev.get("traffic"), "traffic_source": ev.get("traffic_source"),
            "events": {"mean_launch_ms": ev["mean_launch_ms"], "achieved": ev["achieved"], "frac": ev["frac"],
                       "measured_over": ev["measured_over"]},
        }

    line = {
        "metric": METRIC, "value": ms_step, "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": config_of(args.workload, w),
        "variants": other,
        "switch_resid": args.switch_resid,
        "speedup_vs_single_f64": other["single_f64"]["ms"] / ms_step,
        "speedup_vs_double_f64": other["double_f64"]["ms"] / ms_step,
        "roofline": dominant,
        "roofline_events_dominant": dominant_events,
        "roofline_hop_f32": roof32,
        "roofline_hop_f32_dot": roof32d,
        "roofline_hop_f64": roof64,
        "roofline_hop_df": roofdf,
        "roofline_hop_df_dot": roofdfd,
        "roofline_hop_f32_gram": roofg,
        "roofline_hop_f32_alone": roof_alone,
        "roofline_hop_f32_graph": roof_graph,
        "timeline": timeline,
        "stencil_gbs": achieved,
        "e2e": {"value": statistics.mean(e2e_ms), "unit": "ms", "h2d_bytes_per_step": int(b_pin.numel() * 16),
                "d2h_bytes_per_step": int(y_pin.numel() * 16), "rel_err": e2e_err,
                "rel_err_vs_oracle": e2e_err_o},
        "rel_err_vs_oracle": head_vs_oracle,
        "fp32_sweep_shape": {"chosen": ["auto", "wide", "narrow"][tune["shape"]],
                             "ms_per_launch_wide_narrow": tune["times_ms"]},
        "gpu_launches": head_launches // max(1, args.steps),
        "gpu_launches_total_timed": head_launches,
        "clocks": clk,
    }
    # the other configurations of the workload family, measured in the same run:
    # the 32^3 x 64 lattice (l 4, 32 poles) and the 72-system batch
    if not args.no_large:
        try:
            line["variants"]["large_32x32x32x64"] = large_measure(max(1, min(args.steps, 2)), 1)
        except Exception as ex:   # reported, never fatal to the bench line
            line["variants"]["large_32x32x32x64"] = {"error": f"{type(ex).__name__}: {ex}"}
    if not args.no_batched:
        try:
            line["variants"]["batched_72"] = batched_measure(max(1, min(args.steps, 2)), 1, one_at_a_time=False)
        except Exception as ex:
            line["variants"]["batched_72"] = {"error": f"{type(ex).__name__}: {ex}"}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the oracle's own outer-iteration count at the headline's tolerance
        outer_ref, ref_tol = golden_outer_iters(args.workload, tol_h)
        line["cpu_baseline"] = cpu_baseline(w, c, outer_ref or head_res.stats["outer_iters"], ref_tol=ref_tol)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
