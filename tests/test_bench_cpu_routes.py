"""Host helpers of bench.py that time other CPU routes beside the oracle baseline."""
import math

import bench
from synth import lattice_system


def test_sparse_lu_rate_is_bounded_and_positive():
    s = lattice_system((8, 8, 1), 2, "2d", 5)
    v, npoles, t_pole = bench.cpu_sparse_lu_rate(s, -0.1, 0.01, 40, max_seconds=0.2)
    assert v > 0 and 1 <= npoles <= 40 and t_pole > 0
    # the rate is poles x N over the time of a full sweep of M + 1 points
    assert math.isclose(v, 40 * s.n / (t_pole * 41), rel_tol=1e-12)


def test_krylov_oracle_rate_from_time_slices():
    # the iteration rate of bounded slices of column solves, scaled by the iterations a column
    # needs: poles x N / s = M x rate / iterations per column
    s = lattice_system((6, 5, 4), 2, "3d", 6)
    done, t = bench.krylov_slice(s, -0.1, 0.01, 20, 17, 5)
    assert 0 < done <= 21 * 5 and t > 0
    per_col, src = bench.krylov_iterations_per_column(s, -0.1, 0.01, 20, None)
    assert per_col > done / 21 and "convergence" in src
    v, sample, threads = bench.cpu_krylov_rate(s, -0.1, 0.01, 20, None, seconds=0.05, iters_per_task=5)
    assert v > 0 and threads >= 1 and "COCG" in sample


def test_stored_oracle_columns_are_read():
    st = bench.stored_columns("wide", -0.12, 0.01, 40)
    assert st is not None and len(st["columns"]) == 8 and st["leaf_atoms"] == 900
    assert st["bound"] < 1e-10 and st["iterations_per_column"] > 0
    assert len(st["values"]) > 8 * 27 * 8 // 2
    assert bench.stored_columns("wide", -0.12, 0.01, 80) is None
    assert bench.stored_columns("C1", -0.12, 0.01, 40) is None


def test_stored_oracle_counts_are_read():
    import numpy as np
    ref = {0: 1888.610006770609, 9: 13109.959658391954}
    ne = np.zeros(12)
    for i, v in ref.items():
        ne[i] = v + 1e-10
    out = bench._stored_batched_counts(ne, 120, 0.01)
    assert out["systems"] == [0, 1, 2, 4, 5, 6, 8, 9]
    assert out["max_abs_err"] > 1.0                       # the systems left at zero
    assert bench._stored_batched_counts(ne, 80, 0.01) is None


def test_bench_modes_parse():
    import subprocess
    import sys
    out = subprocess.run([sys.executable, "bench.py", "--help"], cwd=bench.ROOT, capture_output=True, text=True)
    assert out.returncode == 0
    for flag in ("--impl", "--config", "--precision", "--energy", "--mu-search", "--eigen", "--no-graph",
                 "--fp64-poles", "--far-ratio", "--leaf"):
        assert flag in out.stdout


def _fake_profile():
    # two schedule steps of the split GEMM and one slicing step, one sweep
    return {"gemm_split:schur": dict(launches=3, ms=30.0, flops=6e12, bytes=3e9, tensor_flops=4e13),
            "gemm_split:sel_t": dict(launches=2, ms=20.0, flops=4e12, bytes=2e9, tensor_flops=2e13),
            "slice:sel_t": dict(launches=2, ms=5.0, flops=0.0, bytes=2e10, tensor_flops=0.0)}


def test_roofline_of_the_dominant_kernel():
    peaks = {"bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0}
    r, kern = bench._roofline(_fake_profile(), 1, peaks, 1.25)
    assert r["kernel"] == "gemm_split" and r["bound"] == "tensor" and r["launches"] == 5
    assert math.isclose(r["achieved"], 6e13 / 0.05 / 1e12) and math.isclose(r["frac"], r["achieved"] / 1700.0)
    assert math.isclose(r["share"], 50.0 / 55.0)
    assert kern["slice"]["launches"] == 2
    # no DRAM figure without a capture of that workload and kernel; the 3D metallic default has one
    assert r["traffic"] is None and "traffic_source" not in r
    r5, _ = bench._roofline(_fake_profile(), 1, peaks, 1.25, ("C5", "split"))
    assert r5["traffic"] == bench.TRAFFIC_PER_LAUNCH[("C5", "split", "gemm_split")]
    assert "ncu" in r5["traffic_source"]
    r2, _ = bench._roofline(_fake_profile(), 1, peaks, 1.25, ("C2", "split"))
    assert r2["traffic"] is None


def test_reference_arm_names_the_workload_like_the_gpu_arm():
    # the driver pairs the two arms by config.workload: both name the lattice and the pole count
    import subprocess
    import sys
    import json
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", "C1", "--steps", "1",
                          "--warmup", "0"], cwd=bench.ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    from synth import config_system
    s = config_system("C1")
    assert line["impl"] == "reference"
    assert line["config"]["workload"] == s.meta["label"] + f", {s.meta['poles']} poles"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["value"] == line["value"]


def test_roofline_of_fp64_and_memory_bound_sweeps():
    peaks = {"bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0}
    # FP64 path: the GEMM counts 8 flops per complex multiply-add, executes 6 (three-multiplication
    # product); achieved is the executed rate against the measured DFMA peak
    prof = {"gemm_f64:schur": dict(launches=4, ms=40.0, flops=4e10, bytes=1e9, tensor_flops=0.0),
            "assemble": dict(launches=1, ms=2.0, flops=0.0, bytes=5e9, tensor_flops=0.0)}
    r, _ = bench._roofline(prof, 1, peaks, 1.25)
    assert r["bound"] == "alu" and r["kernel"] == "gemm_f64" and r["peak"] == 1.25
    assert math.isclose(r["achieved_8flop_count"], 1.0) and math.isclose(r["achieved"], 0.75)
    assert math.isclose(r["frac"], 0.6)
    # an element-wise kernel on top: bytes over time against the measured copy bandwidth
    prof = {"assemble": dict(launches=2, ms=10.0, flops=0.0, bytes=5e10, tensor_flops=0.0)}
    r, _ = bench._roofline(prof, 1, peaks, 1.25)
    assert r["bound"] == "hbm" and math.isclose(r["achieved"], 5000.0) and math.isclose(r["frac"], 5000.0 / 6800.0)
