"""bench.py's JSON line on a small workload (c1: 1e5 rows): the keys of the contract, the
reference arm on the host (the oracle), and the GPU arm with both contexts resident and in
the sequential form (every solver within 1e-9 per block of the binary64 reference, with
every Eq. 5 ratio below 0.1)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _run(*args, timeout=900):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                       text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-3000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    line = _run("--impl", "reference", "--workload", "c1", "--steps", "1", "--warmup", "3")
    assert BASE_KEYS <= set(line)
    assert line["impl"] == "reference" and line["unit"] == "s" and line["higher_is_better"] is False
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["config"]["sample_rows"] == 100_000 and line["config"]["iterations"] > 0
    assert line["e2e"] == {"value": line["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("c1:")


def _check_gpu_line(line):
    assert BASE_KEYS <= set(line)
    assert {"roofline", "clocks", "gpu_launches", "solvers", "kernels"} <= set(line)
    assert line["unit"] == "s" and line["higher_is_better"] is False and line["scaling"] == "weak"
    assert line["value"] > 0 and line["gpu_launches"] > 0
    assert set(line["solvers"]) >= {"fp64_plain", "fp64_jacobi", "mixed", "mixed_jacobi"}
    for name, leg in line["solvers"].items():
        assert leg["final_block_err"] <= 1e-9, (name, leg)
        assert max(leg["eq5_q_max"].values()) <= 0.1, (name, leg)
    best = min(leg["s"] for leg in line["solvers"].values())
    assert abs(line["value"] - best) <= 1e-12 * best
    roof = line["roofline"]
    assert roof["bound"] in ("hbm", "alu") and roof["peak"] > 0 and roof["achieved"] > 0
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-12
    assert {"aprod1_f64", "aprod2_f64", "aprod1_f32", "aprod2_f32", "residual_df",
            "aprod2_f64_on_f32"} <= set(line["kernels"]) <= {"aprod1_f64", "aprod2_f64", "aprod1_f32", "aprod2_f32",
                                                            "residual_df", "aprod2_f64_on_f32", "aprod12_f32"}
    assert "sm_mhz" in line["clocks"]


@pytest.mark.gpu
def test_gpu_arm_line():
    line = _run("--workload", "c1", "--also", "", "--sequential", "no", "--steps", "1", "--warmup", "3",
                "--no-cpu-baseline", "--no-sections")
    _check_gpu_line(line)
    assert line["e2e"]["h2d_bytes_per_step"] > 0 and line["e2e"]["value"] > 0
    assert line["cpu_baseline"] is None and "c2" not in line


@pytest.mark.gpu
def test_gpu_arm_sequential_line():
    line = _run("--workload", "c1", "--also", "", "--sequential", "yes", "--steps", "1", "--warmup", "3",
                "--no-sections")
    _check_gpu_line(line)
    assert line["config"]["contexts"].startswith("binary64 legs first")
    assert line["e2e"]["h2d_bytes_per_step"] > 0 and line["e2e"]["value"] > 0
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] > 0
    assert cpu["single_thread"]["cores"] == 1 and cpu["single_thread"]["value"] > 0


def test_launch_share_model_counts():
    """The benchmark's per-step launch counts (roofline.launch_share_ms) as the launch lists show them:
    the inner iterations as fused passes or as aprod 1 + aprod 2 (the closing iteration that ends each
    inner solve as an aprod 1 alone), one LSQR start per refinement step plus
    one norm pass (the warm start's A^T b pass gives the norms), one aprod 1 for a warm start, one residual
    per step after the first; binary64: one aprod 1 per iteration (+1 warm), iterations + 2 aprod 2."""
    sys.path.insert(0, ROOT)
    import bench

    class G:
        GSR_MIXED = 1

    class E:
        g = G

    t = {"aprod1_f32": 1.0, "aprod2_f32": 10.0, "residual_df": 100.0, "aprod12_f32": 1000.0,
         "aprod1_f64": 1.0, "aprod2_f64": 10.0}
    meta = {"outer": 2, "inner_iterations": [5, 7], "fused": True}
    _, sh = bench.dominant_kernel(E, meta, {"mode": 1, "warm": 1}, t)
    assert sh == {"aprod12_f32": 12000.0, "aprod1_f32": 1.0, "aprod2_f32": 30.0, "residual_df": 100.0}
    meta["fused"] = False
    _, sh = bench.dominant_kernel(E, meta, {"mode": 1}, t)
    assert sh == {"aprod1_f32": 12.0, "aprod2_f32": 150.0, "residual_df": 100.0}
    # closing iterations: the last inner iteration of each refinement step is an aprod 1 alone
    meta = {"outer": 2, "inner_iterations": [5, 7], "fused": True, "closing": True}
    _, sh = bench.dominant_kernel(E, meta, {"mode": 1, "warm": 1}, t)
    assert sh == {"aprod12_f32": 10000.0, "aprod1_f32": 3.0, "aprod2_f32": 30.0, "residual_df": 100.0}
    meta["fused"] = False
    _, sh = bench.dominant_kernel(E, meta, {"mode": 1}, t)
    assert sh == {"aprod1_f32": 12.0, "aprod2_f32": 130.0, "residual_df": 100.0}
    _, sh = bench.dominant_kernel(E, {"iterations": 13}, {"mode": 0, "warm": 2}, t)
    assert sh == {"aprod1_f64": 14.0, "aprod2_f64": 150.0}
