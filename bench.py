#!/usr/bin/env python
"""Benchmark: LSQR time-to-1e-9 on a synthetic Gaia-shaped system on one GB300.

One step = one LSQR solve of the whole system through the library (column
preconditioner, start, iterations in CUDA graphs, unscaling) for the number of
iterations that first brings every block (astro / attitude / instrumental /
global) within 1e-9 relative of a tightly converged reference solution x*.
x* and that iteration count come from untimed solves before the timed region.

Workload (default): 100,000 stars x 200 observations = 2e7 rows, 3,000
attitude knots per axis, 1,000 instrumental unknowns, 1 global, sinusoid
attitude, FP64 values, damp 1e-6 (510,001 unknowns, 4.4 GB of matrix). The
matrix is generated on the device by the seeded generator; it is far larger
than L2 (129 MB), so no L2 flush is needed between timed steps.

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

# algorithmic bytes per row (int32 indices; star_ptr amortised)
BYTES_PER_ROW = {
    ("aprod1", 8): 24 * 8 + 4 + 24 + 16,   # values, knot, 6 instr, y read + write   = 236
    ("aprod2", 8): 24 * 8 + 4 + 24 + 8,    # values, knot, 6 instr, y read           = 228
    ("aprod1", 4): 24 * 4 + 4 + 24 + 16,   # FP32 values, FP64 y                     = 140
    ("aprod2", 4): 24 * 4 + 4 + 24 + 8,    #                                          = 132
}
FLOPS_PER_ROW = 48  # 24 multiply-adds per row in each aprod


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
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
    """nvidia-smi sampling (200 ms) during the timed region."""

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
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
    a = 5 * cfg.n_stars
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
    h = gsrgen.generate(cfg, fp32=w.fp32)
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
            "config": {"workload": f"{args.workload}: {desc(w)}", "solver": "CPU oracle LSQR (FP64, 1 thread)"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": f"oracle LSQR, 1 and 3 iterations on the full system, extrapolated to "
                                       f"{n9} iterations ({note})"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def desc(w):
    c = w.cfg
    return (f"{c.n_stars} stars x {c.obs_min} obs = {c.n_stars * c.obs_min} rows, {c.n_dfa} knots/axis, "
            f"{c.n_instr} instr, {c.n_glob} glob, seed {c.seed}, {'FP32' if w.fp32 else 'FP64'} values, "
            f"damp {w.damp}")


# ---------------------------------------------------------------- our arm
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

    w = gsrgen.workloads()[args.workload]
    cfg = w.cfg
    if world > 1:
        cfg = gsrgen.make_cfg(cfg.seed + 1000 * rank, cfg.n_stars, (cfg.obs_min, cfg.obs_max), cfg.n_dfa, cfg.n_instr,
                              cfg.n_glob, cfg.att_kind, cfg.noise_sigma)
    fp32 = w.fp32
    vdt = torch.float32 if fp32 else torch.float64
    esz = 4 if fp32 else 8

    # ---- system on the device (seeded generator, device twin)
    sp = gsrgen.star_ptr(cfg)
    n = int(sp[-1])
    nc = cfg.ncols()
    spd = torch.tensor(sp, device=dev)
    vals = torch.empty(24 * n, dtype=vdt, device=dev)
    knot = torch.empty(n, dtype=torch.int32, device=dev)
    ins = torch.empty(6 * n, dtype=torch.int32, device=dev)
    gsrgen.dev_rows(cfg, spd, sp, 0, cfg.n_stars, vals, n, knot, ins, stream=sh)
    obs = cfg.obs_min if cfg.obs_min == cfg.obs_max else 0
    ctx = g.Context(cfg.n_stars, obs_per_star=obs, star_ptr=None if obs else sp, n_dfa=cfg.n_dfa,
                    n_instr=cfg.n_instr, n_glob=cfg.n_glob, fp32=fp32, device=local)
    ctx.set_rows(0, n, vals, knot, ins, layout=g.GSR_SOA, plane_stride=n, stream=sh)
    xt = torch.empty(nc, dtype=torch.float64, device=dev)
    gsrgen.dev_xtrue(cfg, xt, stream=sh)
    b = torch.empty(n, dtype=torch.float64, device=dev)
    gsrgen.dev_noise(cfg, b, stream=sh)
    ctx.aprod1(xt, b, stream=sh)  # b = A x_true + eps
    ctx.set_rhs(b, stream=sh)
    torch.cuda.synchronize()

    # host (pinned) copies for the end-to-end leg and the CPU baseline
    host = None
    if not args.no_e2e or (rank == 0 and world == 1 and not args.no_cpu_baseline):
        A_aos = vals.view(24, n).t().contiguous().cpu().pin_memory()
        I_aos = ins.view(6, n).t().contiguous().cpu().pin_memory()
        host = {"A": A_aos, "knot": knot.cpu().pin_memory(), "instr": I_aos, "b": b.cpu().pin_memory()}
    del vals, ins
    torch.cuda.empty_cache()

    solve_kw = dict(damp=w.damp, conlim=0.0)

    # ---- reference solution x* and iterations to 1e-9 (untimed)
    xs = torch.zeros(nc, dtype=torch.float64, device=dev)
    ref_info = ctx.solve(xs, itnlim=20000, atol=1e-15, btol=1e-15, stream=sh, **solve_kw)
    x = torch.zeros(nc, dtype=torch.float64, device=dev)

    def err_at(k):
        ctx.solve(x, itnlim=k, atol=0.0, btol=0.0, stream=sh, **solve_kw)
        torch.cuda.synchronize()
        return max_block_err(x, xs, cfg)

    k = 8
    while err_at(k) > TOL and k < ref_info["itn"]:
        k = int(k * 1.5) + 1
    lo, hi = k // 2, k
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if err_at(mid) <= TOL:
            hi = mid
        else:
            lo = mid
    n9 = hi

    # ---- timed solves (inputs resident)
    for _ in range(args.warmup):
        ctx.solve(x, itnlim=n9, atol=0.0, btol=0.0, stream=sh, **solve_kw)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        ev0.record(stream)
        infos = []
        for _ in range(args.steps):
            infos.append(ctx.solve(x, itnlim=n9, atol=0.0, btol=0.0, stream=sh, **solve_kw))
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms = ev0.elapsed_time(ev1) / args.steps
    final_err = max_block_err(x, xs, cfg)
    t_ms = torch.tensor([ms], device=dev)
    if world > 1:
        dist.barrier()
        dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
    ms = float(t_ms.item())

    # ---- per-kernel timing of aprod1 / aprod2 (same kernels, standalone launches, events on their stream)
    reps = 20
    u = torch.randn(n, dtype=torch.float64, device=dev)
    z = torch.zeros(nc, dtype=torch.float64, device=dev)
    kern = {}
    for name, fn in (("aprod1", lambda: ctx.aprod1(xs, u, stream=sh)), ("aprod2", lambda: ctx.aprod2(u, z, stream=sh))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        kms = e0.elapsed_time(e1) / reps
        gbs = BYTES_PER_ROW[(name, esz)] * n / (kms * 1e-3) / 1e9
        gfl = FLOPS_PER_ROW * n / (kms * 1e-3) / 1e12
        kern[name] = {"ms": kms, "GB/s": gbs, "TFLOP/s": gfl}
    peaks = load_peaks()
    dom = max(kern, key=lambda k: kern[k]["ms"])
    fp64_peak = 1.25  # TFLOP/s, GB300 FP64 (nominal); measured DFMA peak on this machine: ~1.0
    if not fp32:
        roof = {"kernel": dom, "bound": "alu", "achieved": kern[dom]["TFLOP/s"], "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": kern[dom]["TFLOP/s"] / fp64_peak, "traffic": None,
                "peak_src": "nominal FP64 (profiling recipe table)",
                "hbm": {"achieved": kern[dom]["GB/s"], "peak": peaks["hbm_gbs"],
                        "frac": kern[dom]["GB/s"] / peaks["hbm_gbs"], "of": peaks["src"]}}
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": kern[dom]["GB/s"], "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": kern[dom]["GB/s"] / peaks["hbm_gbs"], "traffic": None,
                "peak_src": peaks["src"]}

    # ---- end to end through the C ABI with host buffers (upload + solve + download every step)
    e2e = None
    if not args.no_e2e and host is not None:
        xh = torch.zeros(nc, dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        d2h = xh.numel() * 8
        ctx2 = g.Context(cfg.n_stars, obs_per_star=obs, star_ptr=None if obs else sp, n_dfa=cfg.n_dfa,
                         n_instr=cfg.n_instr, n_glob=cfg.n_glob, fp32=fp32, device=local)

        def e2e_step():
            ctx2.set_system(host["A"], host["knot"], host["instr"], host["b"], stream=sh)
            ctx2.solve(xh, itnlim=n9, atol=0.0, btol=0.0, stream=sh, **solve_kw)

        e2e_step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1) / args.steps
        e2e = {"value": e2e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
        ctx2.close()

    # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and host is not None:
        setup, per_it = oracle_sample(sp, host["A"].numpy(), host["knot"].numpy(), host["instr"].numpy(),
                                      host["b"].numpy(), cfg, w.damp, n9)
        v = setup + per_it * n9
        cpu = {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": f"oracle LSQR (1 thread) for 1 and 3 iterations on the full system, setup + per-iteration "
                         f"time extrapolated to {n9} iterations; host has {cpu_count()} cores"}

    if rank == 0:
        launches_per_step = 5 * n9 + 8  # aprod1, aprod2, colA, scalar, colB per iteration + start/finish kernels
        line = {
            "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if fp32 else "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc(w)}", "solver": "plain LSQR, column-preconditioned",
                       "iterations_to_1e-9": n9, "final_block_err": final_err, "ref_itn": ref_info["itn"],
                       "l2": "inputs larger than L2 (matrix 4.4 GB), no flush", "parallelism": f"replicas x{world}"},
            "kernels": kern, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
            "gpu_launches": launches_per_step * args.steps,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
