#!/usr/bin/env python
"""Benchmark: LSQR time-to-1e-9 on a synthetic Gaia-shaped system on one GB300.

One step = one LSQR solve of the whole system through the library (column
preconditioner, start, iterations in CUDA graphs, unscaling) for the fewest
iterations that bring every block (astro / attitude / instrumental / global)
within 1e-9 relative of a tightly converged binary64 solution x* and keep the
paper's consistency ratio (Sec. 6, Eq. 5) of every unknown against x* below
0.1. x*, and each solver's iteration schedule, come from untimed solves before
the timed region.

Workload (default): the combined-at-scale configuration, 2,000,000 stars x 250
observations = 5e8 rows (1.2e10 nonzeros), 60,000 attitude knots per axis,
20,000 instrumental unknowns, 1 global, sinusoid attitude, damp 1e-6
(10,200,001 unknowns), coefficients rounded to binary32 once so that every
solver solves the identical system. The binary64 legs (binary64 storage,
108 GB) run first; their context is freed before the binary32 one (58 GB) is
built (the two do not fit in device memory together). The headline is the
fastest solver, normally binary32 storage with binary64 refinement from the
learned start; plain binary64 LSQR from x0 = 0 is reported beside it. The
matrix is generated on the device by the seeded generator; it is far larger
than L2 (129 MB), so no L2 flush is needed between timed steps. The 2e7-row
configuration (c2) is measured too and reported under the key "c2".

    python bench.py [--steps K] [--warmup W] [--workload c5] [--impl ours|reference]

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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LSQR s-to-1e-9 (FP64 vs FP32+refine+learned x0), aprod1/2 HBM GB/s, 1 GB300"
TOL = 1e-9   # relative error per block
QTOL = 0.1   # the Eq. 5 ratio of every unknown against x*

# Algorithmic bytes per row of each hot kernel: the row's 24 coefficients, its int32 knot and 6 int32
# instrumental indices, and the row-vector traffic (star_ptr and column vectors amortised). The library
# stores the instrumental indices in 16 bits when n_instr <= 65536 and so moves fewer bytes than this;
# the denominator keeps the int32 indices.
BYTES = {
    "aprod1_f64": 24 * 8 + 28 + 16,      # values, knot + 6 instr, u read + write (binary64)   = 236
    "aprod2_f64": 24 * 8 + 28 + 8,       # values, knot + 6 instr, u read                      = 228
    "aprod1_f32": 24 * 4 + 28 + 8,       # binary32 values, u (binary32) read + write          = 132
    "aprod2_f32": 24 * 4 + 28 + 4,       # binary32 values, u (binary32) read                  = 128
    "residual_df": 24 * 4 + 28 + 8 + 8,  # binary32 values, b (binary64) read, r written       = 140
    # one inner iteration's two products from one read of the tiles (the fused pass): the matrix and the
    # row vector once                                                                         = 132
    "aprod12_f32": 24 * 4 + 28 + 8,
    "aprod2_f64_on_f32": 24 * 4 + 28 + 8,  # binary32 values, binary64 u read                = 132
}
FLOPS_PER_ROW = 48  # 24 multiply-adds per row in each aprod
# DRAM bytes per row of one launch (dram__bytes_read.sum + dram__bytes_write.sum), from single-pass ncu
# captures of the benchmark's standalone launches (bench.py --profile), by the workload whose shape the
# capture had; a launch's traffic is this figure times its rows. Sources under profiles/.
TRAFFIC_PER_ROW = {
    # (the binary64 aprod 2 changed after its 2e7-row capture: no current figure)
    "c2": {"aprod1_f32": 117.4, "aprod2_f32": 120.8, "residual_df": 121.4, "aprod1_f64": 221.4,
           "aprod2_f64": None},   # profiles/traffic_aprod_c2.md
    "c5": {"aprod1_f32": 117.6, "aprod2_f32": 116.7, "residual_df": 121.8, "aprod12_f32": 120.5,
           "aprod1_f64": 221.4, "aprod2_f64": 269.4},  # profiles/traffic_aprod_c5shape.md
}
# the workload each capture stands for (a smaller case of the same shape)
TRAFFIC_SHAPE = {"c2": "c2", "c5": "c5"}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c5")
    ap.add_argument("--also", default="c2",
                    help="a second workload measured after the first and reported under its name ('' for none)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sections", action="store_true",
                    help="skip the section-variant measurement (c2-shaped systems with other row sections)")
    ap.add_argument("--sequential", default="auto", choices=["auto", "yes", "no"],
                    help="one context at a time: the binary64 legs and kernels first, then, after freeing that "
                         "context, the binary32 ones (auto: for the binary32-valued workloads, whose two "
                         "contexts do not fit in device memory together)")
    ap.add_argument("--n-stars", type=int, default=0,
                    help="profiling mode only: override the workload's number of stars (a smaller case for ncu)")
    ap.add_argument("--profile", default=None, choices=["f32", "f64", "mixed", "net"],
                    help="profiling mode for ncu: load the system with binary32 (f32) or binary64 (f64) storage "
                         "and launch each hot kernel --steps times inside an NVTX range 'prof', or (mixed) run the "
                         "default mixed solve from the learned start --steps times; prints timings")
    ap.add_argument("--dfma-probe", action="store_true",
                    help="measure the device's binary64 FMA rate (the ceiling of the binary64 aprods) and exit")
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


def cpu_sample_cfg(gsrgen, cfg, n_stars):
    """A star sample of cfg's shape: its first n_stars stars' worth of rows (same observations per star,
    knots per axis, instrumental and global unknowns, seed and attitude kind)."""
    return gsrgen.make_cfg(cfg.seed, min(n_stars, cfg.n_stars), (cfg.obs_min, cfg.obs_max), cfg.n_dfa, cfg.n_instr,
                           cfg.n_glob, cfg.att_kind, cfg.noise_sigma, n_astro=cfg.n_astro, n_ipr=cfg.n_ipr)


def host_system(gsrgen, oracle, cfg):
    """The oracle's system of cfg (binary32-rounded coefficients widened to binary64, as the GPU solvers
    see them) and its right-hand side b = A x_true + eps; the generator's host twin runs on all cores."""
    h = gsrgen.generate(cfg, fp32=True)
    s = oracle.from_host_system(h)
    return s, oracle.rhs(s, h.x_true, h.eps)


def cpu_baseline(gsrgen, oracle, cfg, damp, n9, full_rows, sample_stars):
    """The oracle timed on the host cores on a star sample of the workload, for the n9 LSQR iterations
    that reach 1e-9 on the full system (the GPU's plain binary64 solver, the same algorithm), scaled to
    the full system by its rows (the work of an iteration is linear in the rows). The single-threaded
    oracle once, the all-cores one (oracle_omp.c) three times (median)."""
    scfg = cpu_sample_cfg(gsrgen, cfg, sample_stars)
    s, b = host_system(gsrgen, oracle, scfg)
    scale = full_rows / s.n_rows
    t0 = time.perf_counter()
    oracle.lsqr(s, b, n9, 0.0, 0.0, 0.0, damp)
    t1 = time.perf_counter() - t0
    tm = []
    for _ in range(3):
        t0 = time.perf_counter()
        oracle.lsqr_omp(s, b, n9, 0.0, 0.0, 0.0, damp)
        tm.append(time.perf_counter() - t0)
    tmed = statistics.median(tm)
    nth = oracle.omp_threads()
    sample = (f"oracle LSQR for the {n9} iterations that reach 1e-9 on the full system, on a star sample of the "
              f"workload ({scfg.n_stars} stars x {cfg.obs_min} obs = {s.n_rows} rows, the workload's "
              f"{cfg.n_dfa} knots/axis and {cfg.n_instr} instrumental unknowns), scaled by rows x{scale:.4g}; "
              f"sample times {tmed:.3f} s ({nth} threads), {t1:.3f} s (1 thread); host has {cpu_count()} cores")
    return {"value": tmed * scale, "unit": "s", "cores": nth, "kind": "oracle", "sample": sample,
            "sample_s": tmed, "single_thread": {"value": t1 * scale, "unit": "s", "cores": 1, "sample_s": t1}}


# ---------------------------------------------------------------- reference arm (the oracle)
REF_SAMPLE_STARS = 18_000  # 4.5e6 rows of the default workload: one oracle solve to 1e-9 in ~6 s


def run_reference(args):
    """The oracle as it stands (single-threaded, binary64) on the host cores. Each step is one whole LSQR
    solve, from x0 = 0 to 1e-9 per block, of a star sample of the workload (its first REF_SAMPLE_STARS
    stars with the full workload's knots and instrumental unknowns): the iteration count that first
    reaches 1e-9 against the oracle's own solution to atol = btol = 1e-15 of the same sample is found
    before the timed steps. The value is the sample's time, not scaled."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import gsrgen
    import oracle

    w = gsrgen.workloads()[args.workload]
    cfg = w.cfg
    scfg = cpu_sample_cfg(gsrgen, cfg, REF_SAMPLE_STARS)
    s, b = host_system(gsrgen, oracle, scfg)
    xs, info_s = oracle.lsqr(s, b, 20000, 1e-15, 1e-15, 0.0, w.damp)

    def err(k):
        x, _ = oracle.lsqr(s, b, k, 0.0, 0.0, 0.0, w.damp)
        worst = 0.0
        for a, z in s.blocks().values():
            if z > a:
                worst = max(worst, np.linalg.norm(x[a:z] - xs[a:z]) / max(np.linalg.norm(xs[a:z]), 1e-3))
        return worst

    hi = 8
    while err(hi) > TOL and hi < info_s["itn"]:
        hi = int(hi * 1.5) + 1
    lo = hi // 2
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if err(mid) <= TOL:
            hi = mid
        else:
            lo = mid
    n9 = hi
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.lsqr(s, b, n9, 0.0, 0.0, 0.0, w.damp)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    v = statistics.median(times)
    scale = (cfg.n_stars * cfg.obs_min) / s.n_rows
    sample = (f"one oracle LSQR solve to 1e-9 per block ({n9} iterations, against the oracle's own solution to "
              f"1e-15, {info_s['itn']} iterations) of a star sample of the workload: {scfg.n_stars} stars x "
              f"{cfg.obs_min} obs = {s.n_rows} rows with its {cfg.n_dfa} knots/axis and {cfg.n_instr} "
              f"instrumental unknowns; the value is the sample's time (the full system has {scale:.4g}x the rows)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc(w)}; coefficients rounded to binary32",
                       "solver": "CPU oracle LSQR (binary64, 1 thread) from x0 = 0",
                       "tolerance": "1e-9 relative per block (astro, attitude, instrumental, global)",
                       "sample_rows": s.n_rows, "iterations": n9},
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample,
                             "scaled_to_workload_s": v * scale},
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
    """Algorithmic bytes per row of a binary32 kernel for the sections of cfg: the row's values, the int32
    knot and instrumental indices, and the row vector (as BYTES for the standard row)."""
    vals = 4 * (cfg.n_astro + 12 + cfg.n_ipr + cfg.n_glob)
    idx = 4 + 4 * cfg.n_ipr
    return vals + idx + {"aprod1_f32": 8, "aprod2_f32": 4, "residual_df": 16}[kernel]


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
def _time_solves(torch, ctx, x, kw, steps, warmup, stream, sh, nvtx=None):
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


class Env:
    """What every measurement shares: torch, the library, the device and its stream, the ranks."""

    def __init__(self, args):
        import torch
        import torch.distributed as dist

        import gsrgen
        import paper_2308_00778_gb300 as g

        self.torch, self.dist, self.gsrgen, self.g = torch, dist, gsrgen, g
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        if self.world > 1:
            dist.init_process_group("nccl")
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        self.stream = torch.cuda.current_stream(self.dev)
        self.sh = self.stream.cuda_stream
        self.peaks = load_peaks()
        self.clk = Clocks(self.local)


def dominant_kernel(env, meta, kw, t):
    """Launches of each hot kernel in one step of a solver times their standalone time: the kernel that
    takes most of the step."""
    g = env.g
    warm_aprod2 = 1 if kw.get("warm") else 0  # the warm start's aprod 1 over the non-astrometric columns
    if kw.get("mode") == g.GSR_MIXED:
        m, its = meta["outer"], sum(meta["inner_iterations"])
        # the first step's residual is b itself (cold) or the warm start's own (its astrometric residual and
        # one aprod 1 over the other columns); the warm start's A^T b pass also gives the column norms, so
        # it stands in for the norm pass (profiles/launches_c5.md)
        n_res = m - 1
        # the last iteration of each inner solve (run to its limit) is a closing one: aprod 1 alone
        closed = m if meta.get("closing") else 0
        if meta.get("fused"):  # the inner iterations take the fused pass; the starts, the norms and A^T b the aprod 2
            share = {"aprod12_f32": (its - closed) * t["aprod12_f32"],
                     "aprod1_f32": (warm_aprod2 + closed) * t["aprod1_f32"],
                     "aprod2_f32": (m + 1) * t["aprod2_f32"], "residual_df": n_res * t["residual_df"]}
        else:
            share = {"aprod1_f32": (its + warm_aprod2) * t["aprod1_f32"],
                     "aprod2_f32": (its - closed + m + 1) * t["aprod2_f32"],
                     "residual_df": n_res * t["residual_df"]}
    else:
        k = meta["iterations"]
        share = {"aprod1_f64": (k + warm_aprod2) * t["aprod1_f64"], "aprod2_f64": (k + 2) * t["aprod2_f64"]}
    return max(share, key=share.get), share


def measure_workload(env, args, name, headline_mode):
    """Every solver on one workload: the schedules that first reach 1e-9 per block with every Eq. 5 ratio
    below 0.1 (untimed), then K timed steps of each after W warm-up steps, the standalone kernels, and
    (headline_mode) the launch count, e2e and CPU baseline of the headline solver."""
    torch, g, gsrgen, dev, stream, sh = env.torch, env.g, env.gsrgen, env.dev, env.stream, env.sh
    from paper_2308_00778_gb300.data import device_system, host_copies

    w = gsrgen.workloads()[name]
    cfg = replica_cfg(gsrgen, w.cfg, env.rank, env.world)
    nc = cfg.ncols()
    damp = w.damp
    seq = args.sequential == "yes" or (args.sequential == "auto" and w.fp32)
    want_e2e = headline_mode and not args.no_e2e
    want_cpu = headline_mode and not args.no_cpu_baseline and env.rank == 0 and env.world == 1

    # ---- one system, coefficients rounded to binary32: every solver sees the same values
    ctx64, _, _ = device_system(cfg, False, True, dev, stream=sh)
    ctx32 = None
    n = ctx64.n_rows

    # ---- the reference solution x* (binary64, tight) and its standard errors (untimed)
    xs = torch.zeros(nc, dtype=torch.float64, device=dev)
    se_ref = torch.zeros(nc, dtype=torch.float64, device=dev)
    ref_info = ctx64.solve(xs, se_out=se_ref, itnlim=20000, atol=1e-15, btol=1e-15, damp=damp, conlim=0.0, stream=sh)
    x = torch.zeros(nc, dtype=torch.float64, device=dev)
    learned = dict(warm=g.GSR_WARM_LEARNED, weights_path=g.WARM_WEIGHTS) if os.path.exists(g.WARM_WEIGHTS) else None
    jacobi = dict(warm=g.GSR_WARM_JACOBI)

    def quality():
        """(the worst block's error / TOL, the worst Eq. 5 ratio / QTOL): a schedule passes when both <= 1"""
        q = eq5_q(x, xs, se_ref, cfg)
        return max(max_block_err(x, xs, cfg) / TOL, max(q.values()) / QTOL)

    def bad(ctx, kw):
        ctx.solve(x, stream=sh, **kw)
        torch.cuda.synchronize()
        return quality()

    def first_k(bad_of, cap):
        k = 8
        while bad_of(k) > 1.0 and k < cap:
            k = int(k * 1.5) + 1
        lo, hi = k // 2, k
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if bad_of(mid) <= 1.0:
                hi = mid
            else:
                lo = mid
        return hi

    def plain_kw(k, warm=None):
        return dict(itnlim=k, atol=0.0, btol=0.0, conlim=0.0, damp=damp, **(warm or {}))

    def mixed_kw(k, m, warm=None, k2=0):
        return dict(mode=g.GSR_MIXED, inner_itn=k, inner_itn_next=k2, max_outer=m, refine_tol=-1.0,
                    inner_tol=1e-30, atol=0.0, btol=0.0, conlim=0.0, damp=damp, **(warm or {}))

    solvers, legs, t = {}, {}, {}

    def time_legs(todo):
        if env.world > 1:
            env.dist.barrier()
        with env.clk:
            for nm, (ctx, kw, meta) in todo.items():
                ms_l, info_l = _time_solves(torch, ctx, x, kw, args.steps, args.warmup, stream, sh, nvtx=f"timed_{nm}")
                q = eq5_q(x, xs, se_ref, cfg)
                solvers[nm] = dict(meta, s=ms_l / 1e3, ms_warm_start=info_l["ms_warm"] if kw.get("warm") else 0.0,
                                   final_block_err=max_block_err(x, xs, cfg), eq5_q_max=q)

    u64 = torch.randn(n, dtype=torch.float64, device=dev)
    z = torch.zeros(nc, dtype=torch.float64, device=dev)

    def time_kernels64():
        t["aprod1_f64"] = _time_kernel(torch, lambda: ctx64.aprod1(xs, u64, stream=sh), stream)
        t["aprod2_f64"] = _time_kernel(torch, lambda: ctx64.aprod2(u64, z, stream=sh), stream)

    cap = ref_info["itn"] + 40
    n9 = first_k(lambda k: bad(ctx64, plain_kw(k)), cap)
    legs["fp64_plain"] = (ctx64, plain_kw(n9), {"iterations": n9, "start": "x0 = 0"})
    for nm, warm in (("fp64_jacobi", jacobi), ("fp64_learned", learned)):
        if warm:
            k = first_k(lambda k, warm=warm: bad(ctx64, plain_kw(k, warm)), cap)
            legs[nm] = (ctx64, plain_kw(k, warm), {"iterations": k, "start": nm.split("_")[1]})
    if seq:  # the binary64 legs and kernels now, then the binary32 context in the binary64 one's place
        time_legs(dict(legs))
        time_kernels64()
        ctx64.close()
        ctx64 = None
        torch.cuda.empty_cache()
    # the binary32 context (and, for e2e, pinned host copies of its rows in the paper's storage)
    ctx32, b32, host = device_system(cfg, True, True, dev, stream=sh, keep_host=want_e2e)
    plan = ctx32.aprod2_plan()  # form 3: the library's inner iterations take the fused pass by default
    fused_inner = plan["passes"] == 3 and FUSED_DEFAULT
    for nm, warm, outers in (("mixed", None, (2, 3)), ("mixed_jacobi", jacobi, (1, 2, 3)),
                             ("mixed_learned", learned, (1, 2, 3))):
        if nm != "mixed" and not warm:
            continue
        cands = []
        for m in outers:
            k = first_k(lambda k, m=m: bad(ctx32, mixed_kw(k, m, warm)), n9 + 20)
            if bad(ctx32, mixed_kw(k, m, warm)) > 1.0:
                continue
            sched = {(k, k)}
            if m > 1:  # a shorter inner limit for the steps after the first
                for k1 in range(max(k - 1, 1), k + 3):
                    if bad(ctx32, mixed_kw(k1, m, warm, k + 2)) > 1.0:
                        continue
                    lo, hi = 0, k + 2
                    while hi - lo > 1:
                        mid = (lo + hi) // 2
                        if bad(ctx32, mixed_kw(k1, m, warm, mid)) <= 1.0:
                            hi = mid
                        else:
                            lo = mid
                    sched.add((k1, hi))
            for k1, k2 in sorted(sched, key=lambda q: q[0] + (m - 1) * q[1])[:3]:
                ms_c, _ = _time_solves(torch, ctx32, x, mixed_kw(k1, m, warm, k2), 2, 1, stream, sh)
                cands.append((ms_c, m, k1, k2))
        if cands:
            _, m, k1, k2 = min(cands)
            legs[nm] = (ctx32, mixed_kw(k1, m, warm, k2),
                        {"outer": m, "inner_iterations": [k1] + [k2] * (m - 1),
                         "start": nm.split("_")[1] if warm else "x0 = 0", "fused": fused_inner,
                         "closing": CLOSE_DEFAULT})

    # ---- timed region: every solver, the same K steps after W warm-up steps each
    time_legs({nm: leg for nm, leg in legs.items() if nm not in solvers})
    headline = min(solvers, key=lambda nm: solvers[nm]["s"])

    # ---- per-kernel timing (the same kernels, standalone launches, CUDA events on their stream)
    u32 = u64.float()
    x32 = xs.float()
    r32 = torch.empty(n, dtype=torch.float32, device=dev)
    if not seq:
        time_kernels64()
    t["aprod1_f32"] = _time_kernel(torch, lambda: ctx32.aprod1_f32(x32, u32, stream=sh), stream)
    t["aprod2_f32"] = _time_kernel(torch, lambda: ctx32.aprod2_f32(u32, z, stream=sh), stream)
    t["residual_df"] = _time_kernel(torch, lambda: ctx32.residual(xs, r32, stream=sh), stream)
    if plan["passes"] == 3:  # the fused pass (y <- A x - 0.5 y, z += A^T y)
        t["aprod12_f32"] = _time_kernel(torch, lambda: ctx32.aprod12_f32(x32, u32, z, -0.5, stream=sh), stream)
    # the mixed refinement's binary64 gradient (used on ill-scaled columns): binary64 aprod 2 on binary32 storage
    u64b = u32.double()
    t["aprod2_f64_on_f32"] = _time_kernel(torch, lambda: ctx32.aprod2(u64b, z, stream=sh), stream)
    del u64b
    shape = TRAFFIC_SHAPE.get(name)
    traffic = TRAFFIC_PER_ROW.get(shape, {}) if shape else {}
    kern = {}
    for kn, kms in t.items():
        bpr = BYTES[kn]
        kern[kn] = {"ms": kms, "GB/s": bpr * n / (kms * 1e-3) / 1e9, "bytes_per_row": bpr,
                    "frac_of_measured_hbm": bpr * n / (kms * 1e-3) / 1e9 / env.peaks["hbm_gbs"],
                    "TFLOP/s": FLOPS_PER_ROW * (2 if kn == "aprod12_f32" else 1) * n / (kms * 1e-3) / 1e12,
                    "ncu_dram_bytes_per_row": traffic.get(kn)}
    hctx, hkw, hmeta = legs[headline]
    dom, share = dominant_kernel(env, hmeta, hkw, t)
    if dom.endswith("f64"):
        dfma = measured_dfma_tflops(env)
        peak = dfma if dfma else 1.25
        roof = {"kernel": dom, "bound": "alu", "achieved": kern[dom]["TFLOP/s"], "peak": peak, "unit": "TFLOP/s",
                "frac": kern[dom]["TFLOP/s"] / peak,
                "traffic": traffic[dom] * n if traffic.get(dom) else None,
                "peak_src": "measured binary64 FMA rate (bench.py --dfma-probe)" if dfma else "nominal FP64"}
    else:
        tr = traffic.get(dom)
        roof = {"kernel": dom, "bound": "hbm", "achieved": kern[dom]["GB/s"], "peak": env.peaks["hbm_gbs"],
                "unit": "GB/s", "frac": kern[dom]["GB/s"] / env.peaks["hbm_gbs"],
                "traffic": tr * n if tr else None, "traffic_unit": "bytes per launch (ncu dram read + write)",
                "algorithmic": kern[dom]["bytes_per_row"] * n, "peak_src": env.peaks["src"],
                "launch_share_ms": share}

    out = {"workload": w, "cfg": cfg, "solvers": solvers, "headline": headline, "kernels": kern, "roofline": roof,
           "ref_info": ref_info, "n9": n9, "learned": learned, "seq": seq}
    if headline_mode:
        # ---- kernel launches of one headline step, counted from the device's activity record (CUPTI)
        out["launches"] = count_launches(torch, lambda: hctx.solve(x, stream=sh, **hkw)) if hctx.h else None
        # ---- end to end through the C ABI from pinned host buffers: upload of the rows and b, solve,
        # download of x, every step (binary32 headline: the binary32 rows; else the binary64 ones)
        if want_e2e and host is not None and hctx is ctx32:
            xh = torch.zeros(nc, dtype=torch.float64).pin_memory()
            up = {k2: v for k2, v in host.items() if k2 != "star_ptr"}
            h2d = sum(v.numel() * v.element_size() for v in up.values())

            def e2e_step():
                ctx32.set_system(up["A"], up["knot"], up["instr"], up["b"], stream=sh)
                ctx32.solve(xh, stream=sh, **hkw)

            ms_e2e = _time_kernel(torch, e2e_step, stream, reps=args.steps)
            out["e2e"] = {"value": ms_e2e / 1e3, "unit": "s", "h2d_bytes_per_step": int(h2d),
                          "d2h_bytes_per_step": int(xh.numel() * 8), "solver": headline}
            del xh, up
        elif want_e2e:
            out["e2e"] = None
        host = None
        # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1 only), a star sample
        if want_cpu:
            import oracle

            out["cpu"] = cpu_baseline(gsrgen, oracle, cfg, damp, n9, n, CPU_SAMPLE_STARS.get(name, cfg.n_stars))
    if ctx64 is not None:
        ctx64.close()
    ctx32.close()
    del xs, se_ref, x, u64, z, u32, x32, r32, b32
    torch.cuda.empty_cache()
    return out


# whether the library's default (gsr_solve_params.inner_fused = 1) runs the inner iterations of a form-3
# system as the fused pass (it does)
FUSED_DEFAULT = True
# whether the library's default (gsr_solve_params.inner_close = 1) ends each inner solve that runs to its
# iteration limit with a closing iteration (aprod 1 and the x update, no aprod 2) (it does)
CLOSE_DEFAULT = True

# stars of the CPU baseline's sample per workload (about 10-30 s of oracle work on the host cores)
CPU_SAMPLE_STARS = {"c5": 80_000, "c3": 100_000, "c2": 100_000}


def measured_dfma_tflops(env):
    """The device's binary64 FMA rate (TFLOP/s, 2 flops per FMA) from the library's probe kernel, or None."""
    try:
        return env.g.dfma_probe_tflops()
    except Exception as e:
        print(f"binary64 FMA probe unavailable: {e!r}", file=sys.stderr)
        return None


def run_ours(args):
    env = Env(args)
    torch, g = env.torch, env.g
    start_activity_record(torch, env.dev)
    main = measure_workload(env, args, args.workload, True)
    w, cfg, solvers, headline = main["workload"], main["cfg"], main["solvers"], main["headline"]
    ms = max_over_ranks(torch, env.dist, solvers[headline]["s"] * 1e3, env.world, env.dev)
    clocks = env.clk.summary()
    extra = None
    if args.also and args.also != args.workload and env.rank == 0 and env.world == 1:
        a = measure_workload(env, args, args.also, False)
        extra = {"workload": f"{args.also}: {desc(a['workload'])}; coefficients rounded to binary32",
                 "headline": a["headline"], "s": a["solvers"][a["headline"]]["s"], "solvers": a["solvers"],
                 "speedup_vs_fp64_plain": {k: a["solvers"]["fp64_plain"]["s"] / v["s"] for k, v in a["solvers"].items()},
                 "kernels": a["kernels"], "roofline": a["roofline"],
                 "reference": f"binary64 LSQR to atol=btol=1e-15 ({a['ref_info']['itn']} itn)"}
    sections = None
    if env.rank == 0 and env.world == 1 and not args.no_sections:
        sections = measure_sections(torch, g, env.gsrgen, env.dev, env.stream, env.sh, env.peaks)
    if env.rank == 0:
        cold = solvers.get("fp64_plain", {}).get("s")
        launches = main.get("launches")
        line = {
            "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": env.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if headline.startswith("mixed") else "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc(w)}; coefficients rounded to binary32",
                       "solver": headline,
                       "reference": f"binary64 LSQR to atol=btol=1e-15 ({main['ref_info']['itn']} itn)",
                       "tolerance": "1e-9 relative per block (astro, attitude, instrumental, global) and Eq. 5 "
                                    "q < 0.1 for every unknown against the reference",
                       "warm_start_weights": os.path.relpath(g.WARM_WEIGHTS, ROOT) if main["learned"] else None,
                       "l2": "inputs larger than L2 (matrix >= 2.4 GB), no flush",
                       "contexts": "binary64 legs first, then the binary32 context in its place" if main["seq"]
                       else "both contexts resident",
                       "parallelism": f"replicas x{env.world}"},
            "solvers": solvers,
            "speedup_vs_fp64_plain": {nm: cold / v["s"] for nm, v in solvers.items()} if cold else None,
            "kernels": main["kernels"], "roofline": main["roofline"], "cpu_baseline": main.get("cpu"),
            "e2e": main.get("e2e"), "clocks": clocks, "sections": sections,
            "gpu_launches": launches * args.steps if launches is not None else None,
        }
        if extra:
            line[args.also] = extra
        print(json.dumps(line), flush=True)
    if env.world > 1:
        env.dist.destroy_process_group()
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
    from paper_2308_00778_gb300.data import device_system

    ctx, b, _ = device_system(cfg, f32, True, dev, stream=sh)
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
        if ctx.aprod2_plan()["passes"] == 3:  # the fused pass (y <- A x - 0.5 y, z += A^T y)
            ops["aprod12_f32"] = lambda: ctx.aprod12_f32(x32, u32, z, -0.5, stream=sh)
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
    gbs = {k: BYTES[k] * n / (v * 1e-3) / 1e9 for k, v in out.items() if k in BYTES}
    print(json.dumps({"profile": args.profile, "workload": args.workload, "rows": n, "n_dfa": cfg.n_dfa,
                      "n_instr": cfg.n_instr, "ms": out, "GB/s": gbs}), flush=True)
    ctx.close()
    return 0


def run_profile_net(args):
    """The warm start's network alone: a forward over the workload's knot series (batch 1) and a training
    step (batch 16 of 2,000 knots), --steps times each inside an NVTX range 'prof'; prints times and the
    achieved dense BF16 rate (2 flops per multiply-add of the six convolutions)."""
    import torch

    import gsrgen
    import paper_2308_00778_gb300 as g

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    L = gsrgen.workloads()[args.workload].cfg.n_dfa
    net = g.Net()
    net.load(g.WARM_WEIGHTS)
    gen = torch.Generator(device=dev)
    gen.manual_seed(0)
    xf = torch.randn((1, L, 6), device=dev, generator=gen)
    out = torch.empty((1, L, 3), device=dev)
    xt = torch.randn((16, 2000, 6), device=dev, generator=gen)
    tt = torch.randn((16, 2000, 3), device=dev, generator=gen)
    ch = [6, 64, 64, 64, 64, 64, 3]
    fl_pos = sum(2 * ci * co * 5 for ci, co in zip(ch[:-1], ch[1:]))  # forward flops per position
    net.forward(xf, out, stream=stream.cuda_stream)
    net.train_step(xt, tt, 0.0, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("prof")
    ms_f = _time_kernel(torch, lambda: net.forward(xf, out, stream=stream.cuda_stream), stream, reps=max(args.steps, 1))
    ms_t = _time_kernel(torch, lambda: net.train_step(xt, tt, 0.0, stream=stream.cuda_stream), stream,
                        reps=max(args.steps, 1))
    torch.cuda.nvtx.range_pop()
    # a training step: forward, backward-data (five layers) and backward-weight, about 3x the forward
    print(json.dumps({"profile": "net", "knots": L, "forward_ms": ms_f,
                      "forward_tflops": fl_pos * L / (ms_f * 1e-3) / 1e12, "train_step_ms": ms_t,
                      "train_step_tflops": 3 * fl_pos * 16 * 2000 / (ms_t * 1e-3) / 1e12}), flush=True)
    net.close()
    return 0


def run_dfma_probe(args):
    import torch

    import paper_2308_00778_gb300 as g

    torch.cuda.set_device(0)
    print(json.dumps({"fp64_fma_tflops": g.dfma_probe_tflops()}), flush=True)
    return 0


def main():
    args = parse_args()
    if args.dfma_probe:
        return run_dfma_probe(args)
    if args.profile == "net":
        return run_profile_net(args)
    if args.profile:
        return run_profile(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
