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
