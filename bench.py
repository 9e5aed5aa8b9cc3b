#!/usr/bin/env python
"""Benchmark: LSQR time-to-1e-9 on a synthetic Gaia-shaped system on one GB300.

One step = one LSQR solve of the whole system through the library (column
preconditioner, start, iterations in CUDA graphs, unscaling) for the number of
iterations that first brings every block (astro / attitude / instrumental /
global) within 1e-9 relative of a tightly converged reference solution x*.
x* and that iteration count come from untimed solves before the timed region.

Workload (default): 100,000 stars x 200 observations = 2e7 rows, 3,000
attitude knots per axis, 1,000 instrumental unknowns, 1 global, sinusoid
attitude, damp 1e-6 (510,001 unknowns). The coefficients are rounded to
binary32 once, so the binary64 solver (binary64 storage, 4.4 GB) and the
mixed solver (binary32 storage, 2.4 GB) solve the identical system; the
headline value is the faster of the two. The matrix is generated on the
device by the seeded generator; it is far larger than L2 (129 MB), so no L2
flush is needed between timed steps.

    python bench.py [--steps K] [--warmup W] [--workload c2] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun each rank solves its own
independent replica of the workload (replicas only: the solve has no
cross-GPU step on one system in this design).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LSQR s-to-1e-9 (FP64 vs FP32+refine+learned x0), aprod1/2 HBM GB/s, 1 GB300"
TOL = 1e-9

# algorithmic bytes per row (int32 knot, 16-bit instrumental columns as stored for n_instr <= 65536;
# star_ptr and column vectors amortised)
BYTES = {
    "aprod1_f64": 24 * 8 + 4 + 12 + 16,   # values, knot, 6 instr, y read + write          = 224
    "aprod2_f64": 24 * 8 + 4 + 12 + 8,    # values, knot, 6 instr, y read                  = 216
    "aprod1_f32": 24 * 4 + 4 + 12 + 8,    # binary32 values, y (binary32) read + write     = 120
    "aprod2_f32": 24 * 4 + 4 + 12 + 4,    # binary32 values, y (binary32) read             = 116
    "residual_df": 24 * 4 + 4 + 12 + 8 + 4,  # values, indices, b (binary64), r write      = 124
}
FLOPS_PER_ROW = 48  # 24 multiply-adds per row in each aprod
# DRAM bytes per row per launch (dram__bytes_read.sum + dram__bytes_write.sum) measured by ncu on the
# 2e7-row workload (one-pass capture of the standalone launches the benchmark times); a launch's traffic is
# this figure times its rows. aprod2_f32 is the max pass and the one-pass star pass with the attitude columns;
# aprod2_f64 the binary64 star pass and the attitude pass.
TRAFFIC_WORKLOAD = "c2"
TRAFFIC_PER_ROW = {"aprod1_f32": 117.3, "aprod2_f32": 120.8, "residual_df": 121.4, "aprod1_f64": 221.4,
                   "aprod2_f64": 275.9}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sections", action="store_true",
                    help="skip the section-variant measurement (c2-shaped systems with other row sections)")
    ap.add_argument("--sequential", action="store_true",
                    help="one context at a time: the binary64 legs and kernels first, then, after freeing that "
                         "context, the binary32 ones (systems whose two contexts do not fit in device memory "
                         "together); no e2e, CPU baseline or section measurement")
    ap.add_argument("--n-stars", type=int, default=0,
                    help="profiling mode only: override the workload's number of stars (a smaller case for ncu)")
    ap.add_argument("--profile", default=None, choices=["f32", "f64", "mixed"],
                    help="profiling mode for ncu: load the system with binary32 (f32) or binary64 (f64) storage "
                         "and launch each hot kernel --steps times inside an NVTX range 'prof', or (mixed) run the "
                         "default mixed solve from the learned start --steps times; prints timings")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback"}


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling (every 50 ms) during the timed region; entering waits for the first sample,
    so that the sampling covers the whole region however long nvidia-smi takes to start."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            n0 = len(self.lines)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.monotonic() + 5.0
            while len(self.lines) == n0 and self.proc.poll() is None and time.monotonic() < deadline:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def block_ranges(cfg):
    a = cfg.n_astro * cfg.n_stars
    t = a + 3 * cfg.n_dfa
    i = t + cfg.n_instr
    return {"astro": (0, a), "att": (a, t), "instr": (t, i), "glob": (i, i + cfg.n_glob)}


def max_block_err(x, ref, cfg):
    import torch

    worst = 0.0
    for a, z in block_ranges(cfg).values():
        if z > a:
            num = torch.linalg.vector_norm(x[a:z] - ref[a:z]).item()
            den = max(torch.linalg.vector_norm(ref[a:z]).item(), 1e-3)
            worst = max(worst, num / den)
    return worst


def eq5_q(x, xr, se, cfg):
    """The paper's consistency ratio (Sec. 6, Eq. 5) of a solution against the binary64 reference,
    q = |x - x_ref| / sqrt(se^2 + se^2) with the reference's standard errors for both; max per section."""
    import torch

    q = (x - xr).abs() / (se * 2.0 ** 0.5).clamp_min(1e-300)
    return {k: float(q[a:z].max()) for k, (a, z) in block_ranges(cfg).items() if z > a}


def cpu_count():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(h_star_ptr, A, knot, instr, b, cfg, damp, n_iter):
    """Time the oracle (single thread) on the full system: 1 and 3 iterations, return
    (setup_s, per_iteration_s)."""
    import oracle

    s = oracle.System(h_star_ptr, A, knot, instr, cfg.n_dfa, cfg.n_instr, cfg.n_glob)
    t0 = time.perf_counter()
    oracle.lsqr(s, b, 1, 0.0, 0.0, 0.0, damp)
    t1 = time.perf_counter()
    oracle.lsqr(s, b, 3, 0.0, 0.0, 0.0, damp)
    t3 = time.perf_counter() - t1
    t1 = t1 - t0
    per_it = max((t3 - t1) / 2.0, 1e-9)
    return max(t1 - per_it, 0.0), per_it


def stored_iterations(workload):
    """Iterations to 1e-9 of the oracle on this workload, when a committed oracle run recorded it."""
    p = os.path.join(ROOT, "tests", "golden", f"{workload}_oracle_itn.json")
    try:
        with open(p) as f:
            return int(json.load(f)["itn_to_1e-9"])
    except Exception:
        return None


# ---------------------------------------------------------------- reference arm (the oracle)
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import gsrgen

    w = gsrgen.workloads()[args.workload]
    cfg = w.cfg
    h = gsrgen.generate(cfg, fp32=True)  # the same binary32-rounded coefficients as the GPU arm
    import oracle

    s = oracle.from_host_system(h)
    b = oracle.rhs(s, h.x_true, h.eps)
    n9 = stored_iterations(args.workload)
    note = "iterations to 1e-9 from tests/golden (oracle run)"
    if n9 is None:
        n9 = 40
        note = "iterations to 1e-9 not recorded; assumed 40"
    times = []
    for i in range(args.warmup + args.steps):
        setup, per_it = oracle_sample(h.star_ptr, h.A, h.knot, h.instr, b, cfg, w.damp, n9)
        if i >= args.warmup:
            times.append(setup + per_it * n9)
    v = statistics.median(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc(w)}; coefficients rounded to binary32",
                       "solver": "CPU oracle LSQR (binary64, 1 thread) from x0 = 0",
                       "tolerance": "1e-9 relative per block (astro, attitude, instrumental, global)"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": f"oracle LSQR, 1 and 3 iterations on the full system, extrapolated to "
                                       f"{n9} iterations ({note})"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def desc(w):
    c = w.cfg
    sec = "" if c.standard else f", sections {c.n_astro} astro / 12 att / {c.n_ipr} instr / {c.n_glob} glob per row"
    return (f"{c.n_stars} stars x {c.obs_min} obs = {c.n_stars * c.obs_min} rows, {c.n_dfa} knots/axis, "
            f"{c.n_instr} instr, {c.n_glob} glob, seed {c.seed}, {'FP32' if w.fp32 else 'FP64'} values, "
            f"damp {w.damp}{sec}")


def variant_bytes(cfg, kernel):
    """Algorithmic bytes per row of a binary32 kernel for the sections of cfg: the row's values, the knot,
    its instrumental columns (16-bit planes up to 65536 unknowns) and the row vector."""
    vals = 4 * (cfg.n_astro + 12 + cfg.n_ipr + cfg.n_glob)
    idx = 4 + cfg.n_ipr * (2 if cfg.n_instr <= 65536 else 4)
    return vals + idx + {"aprod1_f32": 8, "aprod2_f32": 4, "residual_df": 12}[kernel]


def measure_sections(torch, g, gsrgen, dev, stream, sh, peaks, names=("c2g5", "c2a2")):
    """Section variants (Sec. 2, Sec. 4.2) at the benchmark's scale: the binary32 kernels against the HBM
    roofline, and one mixed-precision solve from the learned start with the library's default refinement
    (refine_tol 1e-10) against a tight binary64-arithmetic solve of the same stored values."""
    from paper_2308_00778_gb300.data import device_system

    out = {}
    for name in names:
        w = gsrgen.workloads()[name]
        cfg = w.cfg
        ctx, b, _ = device_system(cfg, True, True, dev, stream=sh)
        n, nc = ctx.n_rows, ctx.n_cols
        xs = torch.zeros(nc, dtype=torch.float64, device=dev)
        ctx.solve(xs, itnlim=20000, atol=1e-15, btol=1e-15, damp=w.damp, conlim=0.0, stream=sh)
        x32 = xs.float()
        u32 = torch.randn(n, dtype=torch.float32, device=dev)
        z = torch.zeros(nc, dtype=torch.float64, device=dev)
        r32 = torch.empty(n, dtype=torch.float32, device=dev)
        t = {"aprod1_f32": _time_kernel(torch, lambda: ctx.aprod1_f32(x32, u32, stream=sh), stream),
             "aprod2_f32": _time_kernel(torch, lambda: ctx.aprod2_f32(u32, z, stream=sh), stream),
             "residual_df": _time_kernel(torch, lambda: ctx.residual(xs, r32, stream=sh), stream)}
        kern = {}
        for k, ms in t.items():
            bpr = variant_bytes(cfg, k)
            gbs = bpr * n / (ms * 1e-3) / 1e9
            kern[k] = {"ms": ms, "GB/s": gbs, "bytes_per_row": bpr, "frac_of_measured_hbm": gbs / peaks["hbm_gbs"]}
        x = torch.zeros(nc, dtype=torch.float64, device=dev)
        kw = dict(mode=g.GSR_MIXED, damp=w.damp, warm=g.GSR_WARM_LEARNED, weights_path=g.WARM_WEIGHTS)
        ms_solve, info = _time_solves(torch, ctx, x, kw, 3, 1, stream, sh)
        out[name] = {"workload": desc(w), "coefficients_per_row": cfg.npar, "kernels": kern,
                     "mixed_learned_default": {"s": ms_solve / 1e3, "outer": info["outer_itn"],
                                               "inner_iterations": info["itn"],
                                               "max_block_err": max_block_err(x, xs, cfg)}}
        ctx.close()
        del xs, x32, u32, z, r32, x, b
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- our arm
def _device_system(g, gsrgen, torch, cfg, fp32_store, round32, dev, sh, keep_host=False):
    from paper_2308_00778_gb300.data import device_system

    return device_system(cfg, fp32_store, round32, dev, stream=sh, keep_host=keep_host)


def _time_solves(torch, ctx, x, kw, steps, warmup, stream, sh, clocks=None, nvtx=None):
    for _ in range(warmup):
        ctx.solve(x, stream=sh, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if nvtx:
        torch.cuda.nvtx.range_push(nvtx)
    e0.record(stream)
    info = None
    for _ in range(steps):
        info = ctx.solve(x, stream=sh, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    if nvtx:
        torch.cuda.nvtx.range_pop()
    return e0.elapsed_time(e1) / steps, info


def _time_kernel(torch, fn, stream, reps=20):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def start_activity_record(torch, dev):
    """A first, empty profiler session: the device's activity record (CUPTI) only sees kernels of the
    library when it was attached before the library's first CUDA work."""
    try:
        from torch.profiler import ProfilerActivity, profile

        with profile(activities=[ProfilerActivity.CUDA]):
            torch.zeros(1, device=dev).add_(1)
            torch.cuda.synchronize()
    except Exception as e:
        print(f"activity record unavailable: {e!r}", file=sys.stderr)


def replica_cfg(gsrgen, cfg, rank, world):
    """Rank r of an N-rank run solves its own replica of the workload: the same shape, seed + 1000 r
    (the solve has no cross-GPU step on one system, so ranks share nothing but the timing)."""
    if world <= 1:
        return cfg
    return gsrgen.make_cfg(cfg.seed + 1000 * rank, cfg.n_stars, (cfg.obs_min, cfg.obs_max), cfg.n_dfa, cfg.n_instr,
                           cfg.n_glob, cfg.att_kind, cfg.noise_sigma, n_astro=cfg.n_astro, n_ipr=cfg.n_ipr)


def max_over_ranks(torch, dist, value, world, device):
    """The largest value over the ranks (the slowest replica's time), after a barrier."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        dist.barrier()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def count_launches(torch, fn):
    """Kernels the device ran during one call of fn, from torch.profiler's CUDA activity record."""
    try:
        from torch.profiler import ProfilerActivity, profile

        fn()
        torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CPU, ProfilerActivity.CUDA]) as prof:
            fn()
            torch.cuda.synchronize()
        n = 0
        kinds = {}
        for ev in prof.events():
            name = ev.name.lower()
            kinds[str(ev.device_type)] = kinds.get(str(ev.device_type), 0) + 1
            if "CUDA" in str(ev.device_type) and "memcpy" not in name and "memset" not in name:
                n += 1
        if not n:
            print(f"launch count unavailable: profiler events by device {kinds}", file=sys.stderr)
        return n or None
    except Exception as e:  # the count is reported as unknown
        print(f"launch count unavailable: {e!r}", file=sys.stderr)
        return None


def run_ours(args):
    import torch
    import torch.distributed as dist

    import gsrgen
    import paper_2308_00778_gb300 as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    start_activity_record(torch, dev)

    w = gsrgen.workloads()[args.workload]
    cfg = replica_cfg(gsrgen, w.cfg, rank, world)
    nc = cfg.ncols()
    damp = w.damp

    # ---- one system, coefficients rounded to binary32; every solver sees the same values
    seq = args.sequential
    if seq:
        args.no_e2e = args.no_cpu_baseline = args.no_sections = True
    ctx64, b64, host = _device_system(g, gsrgen, torch, cfg, False, True, dev, sh, keep_host=False)
    ctx32 = b32 = host = None

    def load32():
        return _device_system(g, gsrgen, torch, cfg, True, True, dev, sh,
                              keep_host=(not args.no_e2e) or (rank == 0 and world == 1 and not args.no_cpu_baseline))

    if not seq:
        ctx32, b32, host = load32()
    n = ctx64.n_rows

    # ---- reference solution x* (binary64, tight) and the schedules that first reach 1e-9 (untimed)
    xs = torch.zeros(nc, dtype=torch.float64, device=dev)
    se_ref = torch.zeros(nc, dtype=torch.float64, device=dev)
    ref_info = ctx64.solve(xs, se_out=se_ref, itnlim=20000, atol=1e-15, btol=1e-15, damp=damp, conlim=0.0,
                           stream=sh)
    x = torch.zeros(nc, dtype=torch.float64, device=dev)
    learned = dict(warm=g.GSR_WARM_LEARNED, weights_path=g.WARM_WEIGHTS) if os.path.exists(g.WARM_WEIGHTS) else None

    def first_k(err, lo_k=1, cap=None):
        k = 8
        cap = cap or ref_info["itn"] + 40
        while err(k) > TOL and k < cap:
            k = int(k * 1.5) + 1
        lo, hi = max(lo_k - 1, k // 2), k
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if err(mid) <= TOL:
                hi = mid
            else:
                lo = mid
        return hi

    def plain_kw(k, warm=None):
        return dict(itnlim=k, atol=0.0, btol=0.0, conlim=0.0, damp=damp, **(warm or {}))

    def mixed_kw(k, m, warm=None, k2=0):
        return dict(mode=g.GSR_MIXED, inner_itn=k, inner_itn_next=k2, max_outer=m, refine_tol=-1.0,
                    inner_tol=1e-30, atol=0.0, btol=0.0, conlim=0.0, damp=damp, **(warm or {}))

    def min_k2(k1, m, warm, hi):
        """Fewest inner iterations of the later refinement steps reaching TOL after k1 in the first (or None)."""
        if err_of(ctx32, mixed_kw(k1, m, warm, hi)) > TOL:
            return None
        lo = 0
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if err_of(ctx32, mixed_kw(k1, m, warm, mid)) <= TOL:
                hi = mid
            else:
                lo = mid
        return hi

    def err_of(ctx, kw):
        ctx.solve(x, stream=sh, **kw)
        torch.cuda.synchronize()
        return max_block_err(x, xs, cfg)

    solvers = {}
    clk = Clocks(local)

    def time_legs(todo):
        if world > 1:
            dist.barrier()
        with clk:
            for name, (ctx, kw, meta) in todo.items():
                ms_l, info_l = _time_solves(torch, ctx, x, kw, args.steps, args.warmup, stream, sh,
                                            nvtx=f"timed_{name}")
                solvers[name] = dict(meta, s=ms_l / 1e3, ms_warm_start=info_l["ms_warm"] if kw.get("warm") else 0.0,
                                     final_block_err=max_block_err(x, xs, cfg), eq5_q_max=eq5_q(x, xs, se_ref, cfg))

    u64 = torch.randn(n, dtype=torch.float64, device=dev)
    z = torch.zeros(nc, dtype=torch.float64, device=dev)
    t = {}

    def time_kernels64():
        t["aprod1_f64"] = _time_kernel(torch, lambda: ctx64.aprod1(xs, u64, stream=sh), stream)
        t["aprod2_f64"] = _time_kernel(torch, lambda: ctx64.aprod2(u64, z, stream=sh), stream)

    # each solver: (context, keyword arguments, description) at the fewest iterations reaching 1e-9
    legs = {}
    n9 = first_k(lambda k: err_of(ctx64, plain_kw(k)))
    legs["fp64_plain"] = (ctx64, plain_kw(n9), {"iterations": n9, "start": "x0 = 0"})
    if learned:
        nl = first_k(lambda k: err_of(ctx64, plain_kw(k, learned)))
        legs["fp64_learned"] = (ctx64, plain_kw(nl, learned), {"iterations": nl, "start": "learned"})
    if seq:  # the binary64 legs and kernels now, then the binary32 context in the binary64 one's place
        time_legs(dict(legs))
        time_kernels64()
        ctx64.close()
        del b64
        torch.cuda.empty_cache()
        ctx32, b32, host = load32()
    for name, warm, outers in (("mixed", None, (2, 3)), ("mixed_learned", learned, (1, 2, 3))):
        if name == "mixed_learned" and not learned:
            continue
        cands = []
        for m in outers:
            k = first_k(lambda k, m=m: err_of(ctx32, mixed_kw(k, m, warm)), cap=n9 + 20)
            if err_of(ctx32, mixed_kw(k, m, warm)) > TOL:
                continue
            sched = {(k, k)}
            if m > 1:  # a shorter inner limit for the steps after the first
                for k1 in range(max(k - 1, 1), k + 3):
                    k2 = min_k2(k1, m, warm, k + 2)
                    if k2 is not None:
                        sched.add((k1, k2))
            for k1, k2 in sorted(sched, key=lambda q: q[0] + (m - 1) * q[1])[:3]:
                ms_c, _ = _time_solves(torch, ctx32, x, mixed_kw(k1, m, warm, k2), 2, 1, stream, sh)
                cands.append((ms_c, m, k1, k2))
        if cands:
            _, m, k1, k2 = min(cands)
            legs[name] = (ctx32, mixed_kw(k1, m, warm, k2),
                          {"outer": m, "inner_iterations": [k1] + [k2] * (m - 1),
                           "start": "learned" if warm else "x0 = 0"})

    # ---- timed region: every solver, the same K steps after W warm-up steps each
    time_legs({nm: leg for nm, leg in legs.items() if nm not in solvers})
    headline = min(solvers, key=lambda nm: solvers[nm]["s"])
    ms = max_over_ranks(torch, dist, solvers[headline]["s"] * 1e3, world, dev)

    # ---- per-kernel timing (same kernels, standalone launches, CUDA events on their stream)
    u32 = u64.float()
    x32 = xs.float()
    r32 = torch.empty(n, dtype=torch.float32, device=dev)
    if not seq:
        time_kernels64()
    t["aprod1_f32"] = _time_kernel(torch, lambda: ctx32.aprod1_f32(x32, u32, stream=sh), stream)
    t["aprod2_f32"] = _time_kernel(torch, lambda: ctx32.aprod2_f32(u32, z, stream=sh), stream)
    t["residual_df"] = _time_kernel(torch, lambda: ctx32.residual(xs, r32, stream=sh), stream)
    traffic = TRAFFIC_PER_ROW if args.workload == TRAFFIC_WORKLOAD else {}
    kern = {}
    for name, kms in t.items():
        bpr = BYTES[name] + (12 if cfg.n_instr > 65536 else 0)  # 32-bit instrumental planes
        kern[name] = {"ms": kms, "GB/s": bpr * n / (kms * 1e-3) / 1e9, "bytes_per_row": bpr,
                      "TFLOP/s": FLOPS_PER_ROW * n / (kms * 1e-3) / 1e12,
                      "ncu_dram_bytes_per_row": traffic.get(name)}
    peaks = load_peaks()
    # launches of each hot kernel in one step of the headline solver (the dominant one is the roofline's)
    hctx, hkw, hmeta = legs[headline]
    warm_aprod2 = 1 if hkw.get("warm") else 0  # A^T b of the warm start (its column norms replace the solve's)
    if hkw.get("mode") == g.GSR_MIXED:
        m, its = hmeta["outer"], sum(hmeta["inner_iterations"])
        n_res = m if hkw.get("warm") else m - 1  # the cold start's first residual is b itself
        share = {"aprod1_f32": its * t["aprod1_f32"], "aprod2_f32": (its + m + 1 + warm_aprod2) * t["aprod2_f32"],
                 "residual_df": n_res * t["residual_df"]}
    else:
        k = hmeta["iterations"]
        share = {"aprod1_f64": (k + (1 if hkw.get("warm") else 0)) * t["aprod1_f64"],
                 "aprod2_f64": (k + 2 + warm_aprod2) * t["aprod2_f64"]}
    dom = max(share, key=share.get)
    if dom.endswith("f64"):
        fp64_peak = 1.25
        roof = {"kernel": dom, "bound": "alu", "achieved": kern[dom]["TFLOP/s"], "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": kern[dom]["TFLOP/s"] / fp64_peak,
                "traffic": traffic[dom] * n if traffic.get(dom) else None,
                "peak_src": "nominal FP64 of the profiling recipe"}
    else:
        tr = traffic.get(dom)
        roof = {"kernel": dom, "bound": "hbm", "achieved": kern[dom]["GB/s"], "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": kern[dom]["GB/s"] / peaks["hbm_gbs"],
                "traffic": tr * n if tr else None, "traffic_unit": "bytes per launch (ncu dram read + write)",
                "algorithmic": kern[dom]["bytes_per_row"] * n, "peak_src": peaks["src"]}

    # ---- kernel launches of one headline step, counted from the device's activity record (CUPTI)
    launches = count_launches(torch, lambda: hctx.solve(x, stream=sh, **hkw)) if hctx.h else None

    # ---- end to end through the C ABI with host buffers (upload + solve + download every step)
    e2e = None
    if not args.no_e2e and host is not None:
        f32 = hctx is ctx32
        xh = torch.zeros(nc, dtype=torch.float64).pin_memory()
        up = {k2: v for k2, v in host.items() if k2 != "star_ptr"}
        if not f32:
            up["A"] = up["A"].double().pin_memory()
        h2d = sum(v.numel() * v.element_size() for v in up.values())
        d2h = xh.numel() * 8
        sp = host["star_ptr"]
        obs = cfg.obs_min if cfg.obs_min == cfg.obs_max else 0
        ctx2 = g.Context(cfg.n_stars, obs_per_star=obs, star_ptr=None if obs else sp, n_dfa=cfg.n_dfa,
                         n_instr=cfg.n_instr, n_glob=cfg.n_glob, fp32=f32, device=local)

        def e2e_step():
            ctx2.set_system(up["A"], up["knot"], up["instr"], up["b"], stream=sh)
            ctx2.solve(xh, stream=sh, **hkw)

        ms_e2e = _time_kernel(torch, e2e_step, stream, reps=args.steps)
        e2e = {"value": ms_e2e / 1e3, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "solver": headline}
        ctx2.close()

    # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and host is not None:
        A64 = host["A"].numpy().astype(np.float64)
        setup, per_it = oracle_sample(host["star_ptr"], A64, host["knot"].numpy(), host["instr"].numpy(),
                                      host["b"].numpy(), cfg, damp, n9)
        v = setup + per_it * n9
        cpu = {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": f"oracle LSQR (1 thread) for 1 and 3 iterations on the full system, setup + per-iteration "
                         f"time extrapolated to the {n9} iterations that reach 1e-9; host has {cpu_count()} cores"}

    # ---- section variants (rank 0, N = 1): kernels and a default mixed solve on c2-shaped variants
    sections = None
    if rank == 0 and world == 1 and not args.no_sections:
        sections = measure_sections(torch, g, gsrgen, dev, stream, sh, peaks)

    if rank == 0:
        cold = solvers.get("fp64_plain", {}).get("s")
        line = {
            "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if headline.startswith("mixed") else "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc(w)}; coefficients rounded to binary32",
                       "solver": headline, "reference": f"binary64 LSQR to atol=btol=1e-15 ({ref_info['itn']} itn)",
                       "tolerance": "1e-9 relative per block (astro, attitude, instrumental, global)",
                       "warm_start_weights": os.path.relpath(g.WARM_WEIGHTS, ROOT) if learned else None,
                       "l2": "inputs larger than L2 (matrix >= 2.4 GB), no flush",
                       "parallelism": f"replicas x{world}"},
            "solvers": solvers,
            "speedup_vs_fp64_plain": {nm: cold / v["s"] for nm, v in solvers.items()} if cold else None,
            "kernels": kern, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
            "sections": sections,
            "gpu_launches": launches * args.steps if launches is not None else None,
        }
        print(json.dumps(line), flush=True)
    ctx64.close()
    ctx32.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_profile(args):
    """A small driver for ncu captures: one context, each hot kernel launched --steps times."""
    import torch

    import gsrgen
    import paper_2308_00778_gb300 as g

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    w = gsrgen.workloads()[args.workload]
    cfg = w.cfg
    if args.n_stars:
        cfg = gsrgen.make_cfg(cfg.seed, args.n_stars, (cfg.obs_min, cfg.obs_max), cfg.n_dfa, cfg.n_instr,
                              cfg.n_glob, cfg.att_kind, cfg.noise_sigma, n_astro=cfg.n_astro, n_ipr=cfg.n_ipr)
    f32 = args.profile in ("f32", "mixed")
    ctx, b, _ = _device_system(g, gsrgen, torch, cfg, f32, True, dev, sh)
    n, nc = ctx.n_rows, ctx.n_cols
    x = torch.randn(nc, dtype=torch.float64, device=dev)
    u = torch.randn(n, dtype=torch.float64, device=dev)
    z = torch.zeros(nc, dtype=torch.float64, device=dev)
    if args.profile == "mixed":
        xm = torch.zeros(nc, dtype=torch.float64, device=dev)
        kw = dict(mode=g.GSR_MIXED, damp=w.damp, warm=g.GSR_WARM_LEARNED, weights_path=g.WARM_WEIGHTS)
        ops = {"mixed_solve": lambda: ctx.solve(xm, stream=sh, **kw)}
    elif f32:
        x32, u32, r32 = x.float(), u.float(), torch.empty(n, dtype=torch.float32, device=dev)
        ops = {"aprod1_f32": lambda: ctx.aprod1_f32(x32, u32, stream=sh),
               "aprod2_f32": lambda: ctx.aprod2_f32(u32, z, stream=sh),
               "residual_df": lambda: ctx.residual(x, r32, stream=sh)}
    else:
        ops = {"aprod1_f64": lambda: ctx.aprod1(x, u, stream=sh), "aprod2_f64": lambda: ctx.aprod2(u, z, stream=sh)}
    for fn in ops.values():  # warm-up outside the profiled range (builds layouts, loads modules)
        fn()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("prof")
    out = {}
    for name, fn in ops.items():
        out[name] = _time_kernel(torch, fn, stream, reps=max(args.steps, 1))
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile": args.profile, "workload": args.workload, "rows": n, "ms": out}), flush=True)
    ctx.close()
    return 0


def main():
    args = parse_args()
    if args.profile:
        return run_profile(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
