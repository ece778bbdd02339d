#!/usr/bin/env python
"""Benchmark: poles x N per second of the selected-inversion density path on one GB300.

Step = one density evaluation rho(mu) (assembly, factor, selected inversion and the residue sum
for every pole of the workload), inputs resident in HBM.  Default workload: the 3D metallic
lattice of 24^3 atoms x 8 orbitals (N = 110592), kT = 0.002 Ha, 160 poles, on the split-precision
path (the largest configuration that fits one GPU); beside it the plain FP64 path is timed on a
stated subset of the poles (every pole costs the same), which gives the split-vs-FP64 speed-up.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ndsi|reference] [--config C5]

Under torchrun the poles are divided among the ranks (ndsi_pole_shard: contiguous ranges, M0 on
one rank); every rank computes its share of Eq. 8 (ndsi_density_poles) and one sum all-reduce
over NCCL of rho and Tr(rho S) completes the step, so N GPUs share one density evaluation
(strong scaling); the max step time over ranks is reported.  `--impl reference` times the CPU
oracle on the same workload, on rank 0 only: the dense generalized eigendecomposition with the
same pole-truncated Fermi function for N <= 8192, else the oracle's Krylov column solves.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "poles x N per second (selected inversion); split-prec vs FP64 speedup at 1e-9"
UNIT = "poles*N/s"
MU = -0.12
DENSE_ORACLE_MAX_N = 8192     # larger systems: the oracle's Krylov column route


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _max_over_ranks(x, dist, world, device):
    """Largest value of x over all ranks (the slowest rank sets the job's time)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(buf, dist, world):
    """In-place sum of a tensor over all ranks: the one exchange of the pole-sharded sweep (each
    rank holds its share of Eq. 8's sum; rho and Tr(rho S) are the totals)."""
    if world > 1:
        dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    return buf


def _job_value(units_per_rank, world, ms_per_step):
    """Whole-job throughput when every rank processes units_per_rank per step (replicas)."""
    return world * units_per_rank / (ms_per_step * 1e-3)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.fh.close()

    def summary(self):
        sms, mx, reasons, watts = [], 0.0, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            rows = [ln.split(",") for ln in open(self.path) if ln.strip()]
        except OSError:
            rows = []
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sms.append(float(r[1]))
                mx = max(mx, float(r[2]))
                watts.append(float(r[3]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_min_mhz": min(sms) if sms else None,
                "sm_max_mhz": mx or None, "reasons": sorted(reasons), "samples": len(sms),
                "power_w_median": statistics.median(watts) if watts else None,
                "power_w_max": max(watts) if watts else None}


# ------------------------------------------------------------------- stored oracle values ---

def stored_columns(name, mu, kT, M):
    """Oracle columns of rho stored by tests/golden/make_rho_columns.py for a workload:
    {"values": {pattern index: rho}, "columns", "bound", "iterations_per_column", "leaf_atoms"},
    or None when no file matches these settings."""
    path = os.path.join(ROOT, "tests", "golden", f"rho_columns_{name}.txt")
    if not os.path.exists(path):
        return None
    out = {"values": {}}
    with open(path) as fh:
        for ln in fh:
            if ln.startswith("#"):
                m = re.search(r"mu = ([-\d.eE+]+), kT = ([-\d.eE+]+), (\d+) poles, leaf_atoms (\d+)", ln)
                if m:
                    out.update(mu=float(m.group(1)), kT=float(m.group(2)), M=int(m.group(3)),
                               leaf_atoms=int(m.group(4)))
                m = re.search(r"# columns: (.*)", ln)
                if m:
                    out["columns"] = [int(c) for c in m.group(1).split()]
                m = re.search(r"a posteriori\): ([\d.eE+-]+);.* (\d+) iterations", ln)
                if m:
                    out["bound"] = float(m.group(1))
                    out["iterations"] = int(m.group(2))
                continue
            k, v = ln.split()
            out["values"][int(k)] = float(v)
    if out.get("mu") != mu or out.get("kT") != kT or out.get("M") != M:
        return None
    out["iterations_per_column"] = out["iterations"] / len(out["columns"])
    return out


# ------------------------------------------------------------------------ CPU baselines ---

def cpu_oracle_rate(system, mu, kT, M, min_seconds=10.0, min_reps=2):
    """Time the oracle's route 1 (dense eigendecomposition + truncated Fermi sum on the pattern);
    also returns the oracle's Tr(rho S) (Eq. 40)."""
    from oracle.dense import generalized_eig, density_eig, on_pattern, electron_count_eig
    Hd, Sd = system.dense()
    times = []
    t_all = time.perf_counter()
    while len(times) < min_reps or time.perf_counter() - t_all < min_seconds:
        t0 = time.perf_counter()
        eps, C = generalized_eig(Hd, Sd)
        on_pattern(density_eig(eps, C, mu, kT, M), system)
        times.append(time.perf_counter() - t0)
        if len(times) >= 20:
            break
    t = statistics.mean(times)
    return M * system.n / t, len(times), t, electron_count_eig(eps, mu, kT, M)


def krylov_slice(system, mu, kT, M, column, iters_per_task):
    """One bounded sample of the oracle's Krylov column route: the M + 1 solves of one column of
    rho (Eq. 8), each advanced by at most iters_per_task COCG iterations.  Returns (iterations
    done, seconds)."""
    import numpy as np
    from oracle.krylov import solve_columns
    from oracle.poles import cf_poles
    z, _ = cf_poles(M)
    alphas = np.concatenate([mu + 1j * z * kT, [1.0 + 0.0j]])
    gammas = np.concatenate([np.ones(M), [0.0]])
    t0 = time.perf_counter()
    _, it, _ = solve_columns(system, alphas, gammas, np.full(M + 1, column), max_iter=iters_per_task,
                             require_converged=False)
    return int(it.sum()), time.perf_counter() - t0


def krylov_iterations_per_column(system, mu, kT, M, stored):
    """COCG iterations one column of rho needs (the stored oracle run's count when there is one,
    else one column solved to convergence now)."""
    if stored is not None:
        return stored["iterations_per_column"], "stored oracle run (tests/golden)"
    from oracle.krylov import density_columns_krylov
    _, info = density_columns_krylov(system, mu, kT, M, [system.n // 2])
    return float(info["iterations"]), "one column solved to convergence"


def cpu_krylov_rate(system, mu, kT, M, stored, seconds=12.0, iters_per_task=12):
    """Throughput of the oracle's Krylov route from bounded samples: the COCG iteration rate of
    time-sliced column solves, divided by the iterations a full column needs (N columns make the
    whole rho): poles x N / s = M x rate / iterations_per_column."""
    from oracle.krylov import krylov_threads
    per_col, src = krylov_iterations_per_column(system, mu, kT, M, stored)
    done, t, reps = 0, 0.0, 0
    while t < seconds or reps < 1:
        d, dt = krylov_slice(system, mu, kT, M, (7919 * (reps + 1)) % system.n, iters_per_task)
        done, t, reps = done + d, t + dt, reps + 1
    rate = done / t
    sample = (f"{reps} time slices of the oracle's Krylov column solves (all {M + 1} points of a "
              f"column, {iters_per_task} COCG iterations each; {done} iterations in {t:.1f} s), scaled "
              f"by the {per_col:.0f} iterations a column of rho needs ({src}) and N = {system.n} columns")
    return M * rate / per_col, sample, krylov_threads()


def cpu_sparse_lu_rate(system, mu, kT, M, max_seconds=10.0):
    """SciPy's sparse LU (SuperLU, COLAMD ordering) of z_p S - H for as many poles as fit in about
    max_seconds, scaled to a full sweep: a lower bound of the cost of a CPU sparse route (the
    selected inversion is not included).  Returns (poles x N per second, poles timed, s per pole)."""
    import numpy as np
    import scipy.sparse
    import scipy.sparse.linalg
    from oracle.poles import cf_poles
    z, _ = cf_poles(M)
    rows = system.rows()
    Hs = scipy.sparse.csc_matrix((system.H, (rows, system.col)), shape=(system.n, system.n))
    Ss = scipy.sparse.csc_matrix((system.S, (rows, system.col)), shape=(system.n, system.n))
    times = []
    t_all = time.perf_counter()
    for zp in z:
        if times and time.perf_counter() - t_all > max_seconds:
            break
        A = ((mu + 1j * zp * kT) * Ss - Hs).tocsc()
        t0 = time.perf_counter()
        scipy.sparse.linalg.splu(A)
        times.append(time.perf_counter() - t0)
    t_pole = float(np.mean(times))
    return M * system.n / (t_pole * (M + 1)), len(times), t_pole


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    from synth import config_system, batched_systems
    if args.config == "C4":
        systems = [s for s in batched_systems() if s.n <= DENSE_ORACLE_MAX_N]
        allsys = batched_systems()
        M, kT = args.poles or 120, 0.01
        label = (f"batched: {M} poles x {len(allsys)} uneven systems "
                 f"(N {min(s.n for s in allsys)}..{max(s.n for s in allsys)})")
        n_total = sum(s.n for s in allsys)
    else:
        system = config_system(args.config)
        systems = [system]
        kT, M = system.meta["kT"], args.poles or system.meta["poles"]
        label, n_total = system.meta["label"] + f", {M} poles", system.n
    cores = os.cpu_count()
    if all(s.n <= DENSE_ORACLE_MAX_N for s in systems):
        from oracle.dense import generalized_eig, density_eig, on_pattern
        dense = [s.dense() for s in systems]

        def step():
            t0 = time.perf_counter()
            for s, (Hd, Sd) in zip(systems, dense):
                eps, C = generalized_eig(Hd, Sd)
                on_pattern(density_eig(eps, C, MU, kT, M), s)
            return M * sum(s.n for s in systems) / (time.perf_counter() - t0)
        kind = "oracle (dense generalized eigendecomposition + pole-truncated Fermi sum)"
        sample = (f"per step one full density evaluation of {len(systems)} system(s) "
                  f"(N = {', '.join(str(s.n) for s in systems)}) by the oracle's route 1")
        if args.config == "C4":
            sample += "; the batched systems with N <= 8192 stand for the whole batch"
    else:
        from oracle.krylov import krylov_threads
        system = systems[0]
        stored = stored_columns(args.config, MU, kT, M)
        per_col, src = krylov_iterations_per_column(system, MU, kT, M, stored)
        counter = [0]

        def step():
            counter[0] += 1
            d, dt = krylov_slice(system, MU, kT, M, (7919 * counter[0]) % system.n, 12)
            return M * (d / dt) / per_col
        cores = krylov_threads()
        kind = "oracle (Krylov column solves of Eq. 8)"
        sample = (f"per step one time slice of the oracle's Krylov solves of a column of rho (all {M + 1} "
                  f"points, 12 COCG iterations each), scaled by the {per_col:.0f} iterations a column "
                  f"needs ({src}) and N = {system.n} columns")
    for _ in range(args.warmup):
        step()
    rates = []
    for _ in range(args.steps):
        rates.append(step())
    # mean time per unit of work over the steps (harmonic mean of the rates)
    value = len(rates) / sum(1.0 / r for r in rates)
    ms = 1e3 * M * n_total / value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": label, "n": n_total, "poles": M, "kT": kT, "mu": MU},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": kind,
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- GPU side ---

def _kernel_totals(prof):
    """Aggregate per-step profiler entries ("gemm_split:schur") into kernels ("gemm_split")."""
    out = {}
    for name, v in prof.items():
        k = name.split(":")[0]
        o = out.setdefault(k, dict(launches=0, ms=0.0, flops=0.0, bytes=0.0, tensor_flops=0.0))
        for f in o:
            o[f] += v[f]
    return out


# DRAM bytes per launch of the dominant kernel (dram__bytes_read.sum + dram__bytes_write.sum,
# averaged over its launches in one sweep) for a workload with default options, from a single-pass
# ncu capture of the same kernel build; an entry is removed whenever the kernel changes.  The 3D
# metallic lattice's entry: every split-GEMM launch of one full-size 8-point chunk (six slices),
# scaled to the sweep's mix of chunks (17 six-slice points, 144 five-slice poles, 21 chunks) in
# proportion to points x slices.
TRAFFIC_PER_LAUNCH = {("C5", "split", "gemm_split"): 3.52e9}
TRAFFIC_SOURCE = {("C5", "split", "gemm_split"):
                  "ncu dram__bytes_read.sum + dram__bytes_write.sum of all 356 split-GEMM launches of "
                  "one 8-point six-slice chunk (4.31 GB per launch), scaled to the sweep's chunk mix; "
                  "algorithmic bytes are ~1.5 GB per launch (operands re-read 2.4x)"}


def _roofline(prof, steps, peaks, fp64_peak, traffic_key=None):
    kern = _kernel_totals(prof)
    dname, d = max(kern.items(), key=lambda kv: kv[1]["ms"])
    total = sum(v["ms"] for v in kern.values())
    if dname == "gemm_split":
        peak = peaks.get("bf16_tflops_sustained", 1729.1)
        achieved = d["tensor_flops"] / (d["ms"] * 1e-3) / 1e12
        r = {"bound": "tensor", "unit": "TFLOP/s", "peak": peak,
             "peak_source": "of measured (MEASURED_PEAKS.json bf16_tflops_sustained; the kernel runs "
                            "inside a long step)",
             "fp64_equivalent_tflops": d["flops"] / (d["ms"] * 1e-3) / 1e12}
    elif dname in ("gemm_f64", "diaginv"):
        peak = fp64_peak
        rate8 = d["flops"] / (d["ms"] * 1e-3) / 1e12
        r = {"bound": "alu", "unit": "TFLOP/s", "peak": peak,
             "peak_source": "of measured (ndsi_fp64_peak in this run: DFMA chains on every SM)"}
        if dname == "gemm_f64":
            # the kernel's algorithm is the three-multiplication complex product: 3 real
            # multiply-adds (6 flops) per complex multiply-add; the conventional count is 8
            achieved = 0.75 * rate8
            r.update(flop_count="6 per complex multiply-add (three-multiplication product, as executed)",
                     achieved_8flop_count=rate8, frac_8flop_count=rate8 / peak)
        else:
            achieved = rate8
            r["flop_count"] = "8 nb^3 per pivot block"
    else:
        peak = peaks.get("hbm_gbs", 6792.7)
        achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
        r = {"bound": "hbm", "unit": "GB/s", "peak": peak,
             "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)"}
    traffic = TRAFFIC_PER_LAUNCH.get(traffic_key + (dname,)) if traffic_key else None
    if traffic is not None:
        r["traffic_source"] = TRAFFIC_SOURCE[traffic_key + (dname,)]
    r.update({"kernel": dname, "achieved": achieved, "frac": achieved / peak, "traffic": traffic,
              "launches": d["launches"], "kernel_ms_per_step": d["ms"] / steps,
              "share": d["ms"] / total})
    return r, kern


def _plan_options(args):
    """Plan options given on the command line (unset ones keep the library defaults)."""
    kw = dict(split_slices=args.slices, outer_block=args.outer, block=args.block, split_bands=args.bands,
              leaf_atoms=args.leaf, split_far_ratio=args.far_ratio)
    return {k: v for k, v in kw.items() if v}


def _autotune(nd, args, plan, H, S, kT, M, n):
    """Per-step tensor-core / FP64 choice of a split plan, made once before any timing: on every
    pole of small systems, on ten poles (one workspace chunk) of large ones."""
    if args.no_autotune:
        return None
    m = M if n <= 20000 else min(M, 10)
    n_split, n_fp64 = nd.ndsi_autotune(plan, H, S, MU, kT, m)
    shapes = nd.ndsi_plan_export(plan, "tile_shapes")
    widths = {int(w): int((shapes == w).sum()) for w in sorted(set(shapes.tolist())) if w > 0}
    return {"tensor_core_steps": n_split, "fp64_steps": n_fp64, "poles_timed": m,
            "tensor_steps_by_tile_columns": widths,
            "launches_per_pole_batch": int(nd.ndsi_plan_info(plan)["n_launches"])}


def _timed_steps(torch, step, stream, flush, steps, ahead):
    """L2 flush, start event, step, end event per step on the launch stream; with `ahead` the
    steps are enqueued back to back, else synchronised one by one.  Returns ms per step."""
    events = []
    torch.cuda.synchronize()
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        events.append((e0, e1))
        if not ahead:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in events]


def _measure(nd, torch, plan, step, steps, warmup, stream, flush, prof_steps, by_level=False):
    """Time `steps` density sweeps as the library runs them (one captured CUDA graph per sweep),
    then repeat `prof_steps` of them with direct launches and per-launch CUDA events for the
    kernel breakdown."""
    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    # the timed region alone is what `ncu --profile-from-start off` records (a no-op otherwise)
    torch.cuda.profiler.start()
    times = _timed_steps(torch, step, stream, flush, steps, True)
    torch.cuda.profiler.stop()
    nd.ndsi_profile_enable(plan, True, by_level=by_level)
    prof_times = _timed_steps(torch, step, stream, flush, prof_steps, False)
    prof = nd.ndsi_profile_read(plan)
    nd.ndsi_profile_enable(plan, False)
    return times, prof, prof_times


def _parity(args, system, rho, kT, M, stored, e_buf=None):
    """max |rho - oracle| on sampled columns: the stored oracle columns of the workload when
    present, else the oracle's column route run now (SuperLU solves per pole)."""
    import numpy as np
    if stored is not None:
        idx = np.fromiter(stored["values"].keys(), dtype=np.int64)
        ref = np.fromiter(stored["values"].values(), dtype=np.float64)
        err = float(np.max(np.abs(rho[idx] - ref)))
        return {"max_abs_err_rho": err, "columns": stored["columns"], "entries": int(idx.size),
                "oracle": "stored Krylov columns of Eq. 8 (tests/golden, oracle-only script)",
                "oracle_error_bound": stored["bound"],
                "tolerance": 1e-10 if args.precision == "fp64" else 1e-9}
    if system.n > 20000:
        return {"skipped": "no stored oracle columns for these settings (the column route takes "
                           "hours at this size; tests/golden/make_rho_columns.py stores them)"}
    from oracle.dense import density_columns
    rng = np.random.default_rng(11)
    cols = sorted(rng.choice(system.n, 3, replace=False).tolist())
    ref = density_columns(system, MU, kT, M, cols)
    rows = system.rows()
    err = 0.0
    for t_, j in enumerate(cols):
        sel = np.nonzero(system.col == j)[0]
        err = max(err, float(np.max(np.abs(rho[sel] - ref[rows[sel], t_]))))
    out = {"max_abs_err_rho": err, "columns": cols, "oracle": "SuperLU columns of Eq. 8, run now",
           "tolerance": 1e-10 if args.precision == "fp64" else 1e-9}
    if e_buf is not None:
        from oracle.dense import energy_density_columns
        eref = energy_density_columns(system, MU, kT, M, cols)
        ee = 0.0
        for t_, j in enumerate(cols):
            sel = np.nonzero(system.col == j)[0]
            ee = max(ee, float(np.max(np.abs(e_buf[sel] - eref[rows[sel], t_]))))
        out["max_abs_err_energy_density"] = ee
    return out


def _release(torch):
    """Drop unreferenced plans (their device workspaces) before the next plan is sized."""
    import gc
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _other_leg(nd, torch, args, system, H, S, kT, M, stream, flush, prec_code, fp64_peak, ms_main,
               rho_main, ne_main):
    """The other precision on the same workload.  Every pole costs the same, so a large system's
    FP64 path is timed on a stated subset of the poles and compared per contour point; the two
    paths' rho are compared on that subset's expansion.  One plan (and its workspace) is alive at
    a time, so each gets the device memory the headline plan had."""
    import numpy as np
    _release(torch)
    oprec = "split" if args.precision == "fp64" else "fp64"
    Mo = M if system.n <= 20000 else min(M, args.fp64_poles or 8)
    kw = _plan_options(args)
    plan2 = nd.analyze_system(system, precision=prec_code[oprec], **kw)
    tune2 = _autotune(nd, args, plan2, H, S, kT, M, system.n) if oprec == "split" else None
    rho2 = torch.zeros(system.nnz, dtype=torch.float64, device=H.device)
    ne2 = torch.zeros(1, dtype=torch.float64, device=H.device)

    def step2():
        nd.ndsi_density(plan2, H, S, MU, kT, Mo, rho2, ne2, stream=stream)
    w2, k2 = (max(args.warmup, 3), args.steps) if Mo == M else (1, 1)
    t2, prof2, _ = _measure(nd, torch, plan2, step2, k2, w2, stream, flush, 1)
    ms2 = sum(t2) / len(t2)
    rl2, kk2 = _roofline(prof2, 1, _peaks(), fp64_peak)
    per_point_main = ms_main / (M + 1)
    per_point_other = ms2 / (Mo + 1)
    split_pp, fp64_pp = ((per_point_other, per_point_main) if oprec == "split" else
                         (per_point_main, per_point_other))
    out = {"precision": oprec, "poles": Mo, "ms_per_step": ms2, "steps": k2, "warmup": w2,
           "ms_per_point": per_point_other, "value": Mo * system.n / (ms2 * 1e-3),
           "split_speedup_vs_fp64": fp64_pp / split_pp, "autotune": tune2, "roofline": rl2,
           "kernels": {k: {"launches": v["launches"], "ms_per_step": v["ms"]} for k, v in kk2.items()}}
    rho2_h = rho2.cpu().numpy()
    ne2_h = float(ne2.cpu()[0])
    del plan2, step2
    _release(torch)
    if Mo == M:
        out["max_abs_rho_diff_vs_headline"] = float(np.max(np.abs(rho2_h - rho_main)))
        out["abs_n_elec_diff_vs_headline"] = abs(ne2_h - ne_main)
    else:
        # both precisions on the subset's expansion (Mo poles)
        plan_main = nd.analyze_system(system, precision=prec_code[args.precision], **kw)
        rho3 = torch.zeros_like(rho2)
        ne3 = torch.zeros_like(ne2)
        nd.ndsi_density(plan_main, H, S, MU, kT, Mo, rho3, ne3, stream=stream)
        torch.cuda.synchronize()
        out["max_abs_rho_diff_same_poles"] = float(np.max(np.abs(rho2_h - rho3.cpu().numpy())))
        out["fp64_ms_per_step_full_poles_estimate"] = (fp64_pp * (M + 1))
        out["note"] = (f"the FP64 path is timed on the first {Mo} poles (+ M0): every pole of one "
                       "system costs the same, so the speed-up is the ratio of the two paths' time "
                       "per contour point")
        del plan_main
        _release(torch)
    return out, (fp64_pp * (M + 1))


def _lattice_system(spec):
    """A 3D cubic lattice NXxNYxNZxO (cut-off 1.8a, the workloads' recipe), kT 0.01, 40 poles: a
    profiling workload with chosen front sizes (with --leaf)."""
    from synth import SEED_BASE, lattice_system
    nx, ny, nz, o = (int(v) for v in spec.lower().split("x"))
    s = lattice_system((nx, ny, nz), o, "3d", SEED_BASE + 9)
    s.meta.update(name=spec, kT=0.01, poles=40,
                  label=f"3D cubic {nx}x{ny}x{nz} atoms x {o} orbitals (N={s.n})")
    return s


def run_ndsi(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1005_0088_gb300.build import build
    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
    import paper_1005_0088_gb300 as nd
    from synth import config_system

    prec_code = {"fp64": nd.NDSI_PREC_FP64, "split": nd.NDSI_PREC_SPLIT}
    if args.config == "C4":
        return run_batched(args, nd, torch, dist, rank, world, local, prec_code)
    system = _lattice_system(args.lattice) if args.lattice else config_system(args.config)
    kT, M = system.meta["kT"], system.meta["poles"]
    if args.poles:
        M = args.poles
    stored = None if args.lattice else stored_columns(args.config, MU, kT, M)
    plan = nd.analyze_system(system, precision=prec_code[args.precision], **_plan_options(args))
    info = nd.ndsi_plan_info(plan)
    dev = torch.device("cuda", local)
    fp64_peak = nd.ndsi_fp64_peak()
    H = torch.as_tensor(system.H, device=dev)
    S = torch.as_tensor(system.S, device=dev)
    tune = _autotune(nd, args, plan, H, S, kT, M, system.n)
    if args.no_graph:
        nd.ndsi_graph_enable(plan, False)
    nnz = system.nnz
    out = torch.zeros(nnz + 1, dtype=torch.float64, device=dev)    # rho, then Tr(rho S)
    rho, ne = out[:nnz], out[nnz:]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()
    pb, pe, m0 = nd.ndsi_pole_shard(M, rank, world)
    e_buf = torch.zeros_like(rho) if args.energy else None

    def step():
        if world == 1:
            if e_buf is None:
                nd.ndsi_density(plan, H, S, MU, kT, M, rho, ne, stream=stream)
            else:
                nd.ndsi_density_energy(plan, H, S, MU, kT, M, rho, e_buf, ne, stream=stream)
        else:
            nd.ndsi_density_poles(plan, H, S, MU, kT, M, pb, pe, m0, rho, ne, stream=stream)
            _sum_over_ranks(out, dist, world)

    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        times, prof, prof_times = _measure(nd, torch, plan, step, args.steps, args.warmup, stream, flush,
                                           min(args.steps, 2), by_level=args.by_level)
        graph_nodes = nd.ndsi_graph_info(plan)
    if world > 1:
        dist.barrier()
    total_ms = _max_over_ranks(sum(times), dist, world, dev)
    ms_step = total_ms / args.steps
    value = M * system.n / (ms_step * 1e-3)       # one density evaluation per step, all ranks
    rho_main = rho.cpu().numpy()
    ne_main = float(ne.cpu()[0])
    # end to end through the public API with pinned host buffers (copies inside the call)
    Hh = torch.as_tensor(system.H).pin_memory()
    Sh = torch.as_tensor(system.S).pin_memory()
    out_h = torch.zeros(nnz + 1, dtype=torch.float64).pin_memory()
    rho_h, ne_h = out_h[:nnz], out_h[nnz:]

    def e2e_step():
        if world == 1:
            nd.ndsi_density(plan, Hh, Sh, MU, kT, M, rho_h, ne_h, stream=stream)
        else:
            nd.ndsi_density_poles(plan, Hh, Sh, MU, kT, M, pb, pe, m0, rho, ne, stream=stream)
            _sum_over_ranks(out, dist, world)
            out_h.copy_(out)
    e2e_step()
    e2e_steps = min(args.steps, 3)
    e2e_times = []
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = _max_over_ranks(sum(e2e_times) / len(e2e_times), dist, world, dev)
    sys.stderr.write(json.dumps({"progress": "headline timed", "ms_per_step": ms_step,
                                 "e2e_s": e2e_s, "step_ms": times}) + "\n")
    # the other precision on the same workload: split-vs-FP64 speedup and rho difference
    other, fp64_ms_full = None, None
    del plan, step, e2e_step              # the headline plan's workspace goes back to the device
    if not args.no_other and rank == 0:
        other, fp64_ms_full = _other_leg(nd, torch, args, system, H, S, kT, M, stream, flush, prec_code,
                                         fp64_peak, ms_step * world if world > 1 else ms_step, rho_main,
                                         ne_main)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    default_opts = not (args.poles or args.outer or args.block or args.slices or args.bands or args.leaf
                        or args.far_ratio)
    roofline, kern = _roofline(prof, len(prof_times), _peaks(), fp64_peak,
                               (args.config, args.precision) if default_opts else None)
    launches = sum(v["launches"] for v in kern.values())
    parity = None if args.no_parity else _parity(args, system, rho_main, kT, M, stored,
                                                 e_buf.cpu().numpy() if e_buf is not None else None)
    cpu = None
    n_elec = {"value": ne_main}
    golden = os.path.join(ROOT, "tests", "golden", "c3_electron_count.txt")
    if args.config == "C3" and M == 80 and os.path.exists(golden):
        # the oracle's count for this workload (eigenvalues by LAPACK, stored by
        # tests/golden/make_c3_electron_count.py): too slow to recompute inside the bench
        with open(golden) as fh:
            ne_ref = float([ln for ln in fh if ln.strip() and not ln.startswith("#")][0])
        n_elec.update(oracle=ne_ref, abs_err=abs(ne_main - ne_ref), oracle_source="stored (oracle eigenvalues)")
    if world == 1 and not args.no_cpu:
        if system.n <= DENSE_ORACLE_MAX_N:
            v, reps, t_rep, ne_oracle = cpu_oracle_rate(system, MU, kT, M)
            n_elec.update(oracle=ne_oracle, abs_err=abs(ne_main - ne_oracle))
            cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"{reps} full density evaluations of the workload by dense generalized "
                             f"eigendecomposition + {M}-pole Fermi sum ({t_rep:.2f} s each)"}
        elif stored is not None or system.n <= 20000:
            v, sample, threads = cpu_krylov_rate(system, MU, kT, M, stored)
            cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}
        if cpu is not None and system.n <= 16384:
            vs, npl, tpl = cpu_sparse_lu_rate(system, MU, kT, M)
            cpu["other_cpu_routes"] = {
                "scipy_sparse_lu": {"value": vs, "unit": UNIT, "cores": os.cpu_count(),
                                    "sample": f"SuperLU factorisation of {npl} poles, {tpl * 1e3:.1f} ms "
                                              f"each, scaled to {M + 1} points; factorisation only (no "
                                              "selected inversion), a lower bound of a CPU sparse route"}}
    speedup = other["split_speedup_vs_fp64"] if other else None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else f"bf16x{info['split_slices']}->f64",
            "data": "synthetic",
            "split_speedup_vs_fp64": speedup,
            "fp64_ms_per_step": (ms_step if args.precision == "fp64" else fp64_ms_full),
            "max_abs_err_rho_vs_oracle": parity.get("max_abs_err_rho") if parity else None,
            "config": {"workload": system.meta["label"] + f", {M} poles"
                                   + (", rho and energy density matrix" if args.energy else ""),
                       "n": system.n, "poles": M, "kT": kT, "mu": MU, "nnz": nnz,
                       "precision": args.precision, "split_slices": info["split_slices"],
                       "split_bands": info["split_bands"],
                       "l2": "flushed (256 MB write) before every timed step; inputs and fronts "
                             "are far larger than L2",
                       "flops_per_pole": info["flops_per_pole"],
                       "parallelism": "one GPU" if world == 1 else f"pole-sharded x{world} (sum all-reduce of rho)"},
            "e2e": {"value": M * system.n / e2e_s, "unit": UNIT, "steps": e2e_steps,
                    "h2d_bytes_per_step": 2 * 8 * nnz,
                    "d2h_bytes_per_step": 8 * nnz + 8},
            "gpu_launches": launches // len(prof_times) * args.steps,
            "step_ms": [round(t, 4) for t in times],
            "autotune": tune, "fp64_peak_tflops_measured": fp64_peak,
            "graph": {"kernel_nodes": graph_nodes,
                      "ms_per_step_direct_launches": sum(prof_times) / len(prof_times),
                      "note": "timed steps replay one captured CUDA graph per sweep; the kernel "
                              "breakdown and roofline come from steps repeated with direct launches "
                              "bracketed by CUDA events on the launch stream"},
            "roofline": roofline, "clocks": clk.summary(), "cpu_baseline": cpu,
            "parity": parity, "n_elec": n_elec, "other_precision": other,
            "kernels": {k: {"launches": v["launches"] // len(prof_times),
                            "ms_per_step": v["ms"] / len(prof_times),
                            "gbs": v["bytes"] / max(v["ms"], 1e-9) / 1e6,
                            "tflops": v["flops"] / max(v["ms"], 1e-9) / 1e9}
                        for k, v in kern.items()},
            "steps_detail": {k: {"launches": v["launches"] // len(prof_times),
                                 "ms_per_step": v["ms"] / len(prof_times)}
                             for k, v in prof.items()}}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def _stored_batched_counts(ne, M, kT):
    """Tr(rho S) of the batched systems against the oracle's eigenvalue counts stored by
    tests/golden/make_c4_electron_counts.py (systems with N <= 16384, mu -0.12, kT 0.01, 120
    poles), or None for other settings."""
    path = os.path.join(ROOT, "tests", "golden", "c4_electron_counts.txt")
    if M != 120 or kT != 0.01 or MU != -0.12 or not os.path.exists(path):
        return None
    with open(path) as fh:
        ref = {int(l.split()[0]): float(l.split()[2]) for l in fh if l.strip() and not l.startswith("#")}
    return {"systems": sorted(ref), "max_abs_err": max(abs(float(ne[i]) - v) for i, v in ref.items()),
            "source": "stored (oracle eigenvalues)"}


def run_batched(args, nd, torch, dist, rank, world, local, prec_code):
    """C4: twelve uneven systems (1D/2D/3D, N 2048..32768) in one batched plan, 120 poles."""
    import numpy as np
    from synth import batched_systems
    systems = batched_systems()
    M = args.poles or 120
    kT = 0.01
    plan = nd.analyze_batched(systems, precision=prec_code[args.precision], **_plan_options(args))
    info = nd.ndsi_plan_info(plan)
    dev = torch.device("cuda", local)
    H = torch.as_tensor(np.concatenate([s.H for s in systems]), device=dev)
    S = torch.as_tensor(np.concatenate([s.S for s in systems]), device=dev)
    nnz = int(H.shape[0])
    out = torch.zeros(nnz + len(systems), dtype=torch.float64, device=dev)   # rho, then Tr(rho S) per system
    rho, ne = out[:nnz], out[nnz:]
    mus = np.full(len(systems), MU)
    kts = np.full(len(systems), kT)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    pb, pe, m0 = nd.ndsi_pole_shard(M, rank, world)

    def step():
        if world == 1:
            nd.ndsi_density_batched(plan, H, S, mus, kts, M, rho, ne, stream=stream)
        else:
            # (pole, system) pairs split by pole: every rank its pole range of all systems
            nd.ndsi_density_batched_poles(plan, H, S, mus, kts, M, pb, pe, m0, rho, ne, stream=stream)
            _sum_over_ranks(out, dist, world)
    for _ in range(max(args.warmup, 3)):
        step()

    def timed_steps():
        out = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return out
    with ClockSampler(local) as clk:
        torch.cuda.profiler.start()
        times = timed_steps()
        torch.cuda.profiler.stop()
    graph_nodes = nd.ndsi_graph_info(plan)
    nd.ndsi_profile_enable(plan, True)
    prof_times = timed_steps()
    prof = nd.ndsi_profile_read(plan)
    nd.ndsi_profile_enable(plan, False)
    ms = _max_over_ranks(sum(times), dist, world, dev) / len(times)
    ntot = sum(s.n for s in systems)
    # end to end through the public API with pinned host buffers (copies inside the call)
    Hh = H.cpu().pin_memory()
    Sh = S.cpu().pin_memory()
    rho_h = torch.zeros(nnz, dtype=torch.float64).pin_memory()
    ne_h = torch.zeros(len(systems), dtype=torch.float64).pin_memory()
    out_h = torch.zeros(nnz + len(systems), dtype=torch.float64).pin_memory()

    def e2e_step():
        if world == 1:
            nd.ndsi_density_batched(plan, Hh, Sh, mus, kts, M, rho_h, ne_h, stream=stream)
        else:
            nd.ndsi_density_batched_poles(plan, Hh, Sh, mus, kts, M, pb, pe, m0, rho, ne, stream=stream)
            _sum_over_ranks(out, dist, world)
            out_h.copy_(out)
    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_step()
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks(time.perf_counter() - t0, dist, world, dev)
    # parity outside the timed region: sampled columns of the three smallest systems by sparse
    # solves per pole (the oracle's column route)
    parity = None
    if not args.no_parity and rank == 0:
        from oracle.dense import density_columns
        rho_all = rho.cpu().numpy()
        offs = np.cumsum([0] + [s_.nnz for s_ in systems])
        rng = np.random.default_rng(12)
        err, checked = 0.0, []
        for i in sorted(range(len(systems)), key=lambda i: systems[i].n)[:3]:
            sy = systems[i]
            cols = sorted(rng.choice(sy.n, 2, replace=False).tolist())
            ref = density_columns(sy, MU, kT, M, cols)
            rows = sy.rows()
            r_i = rho_all[offs[i]:offs[i + 1]]
            for t_, j in enumerate(cols):
                sel = np.nonzero(sy.col == j)[0]
                err = max(err, float(np.max(np.abs(r_i[sel] - ref[rows[sel], t_]))))
            checked.append({"system": i, "n": sy.n, "columns": cols})
        parity = {"max_abs_err_rho": err, "checked": checked,
                  "tolerance": 1e-10 if args.precision == "fp64" else 1e-9}
    roofline, kern = _roofline(prof, args.steps, _peaks(), nd.ndsi_fp64_peak())
    line = {"metric": METRIC, "value": M * ntot / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else f"bf16x{info['split_slices']}->f64", "data": "synthetic",
            "config": {"workload": f"batched: {M} poles x {len(systems)} uneven systems "
                                   f"(N {min(s.n for s in systems)}..{max(s.n for s in systems)})",
                       "schedule": "one plan, one launch per tree level and step",
                       "n_total": ntot, "poles": M, "kT": kT, "nnz": nnz, "precision": args.precision,
                       "flops_per_pole": info["flops_per_pole"], "n_levels": info["n_levels"],
                       "l2": "flushed (256 MB write) before every timed step"},
            "e2e": {"value": M * ntot / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": 2 * 8 * nnz, "d2h_bytes_per_step": 8 * nnz + 8 * len(systems)},
            "gpu_launches": sum(v["launches"] for v in kern.values()),
            "graph": {"kernel_nodes": graph_nodes,
                      "ms_per_step_direct_launches": sum(prof_times) / len(prof_times)},
            "roofline": roofline, "clocks": clk.summary(),
            "n_elec": ne.cpu().numpy().tolist(),
            "n_elec_oracle": _stored_batched_counts(ne.cpu().numpy(), M, kT),
            "parity": parity,
            "kernels": {k: {"launches": v["launches"] // args.steps, "ms_per_step": v["ms"] / args.steps}
                        for k, v in kern.items()}}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_mu_search_batched(args, nd, torch):
    """Chemical-potential search for all twelve systems of the batched workload at once
    (ndsi_find_mu_batched: lockstep searches, one batched sweep per round, procedure (2) start):
    batched sweeps and wall time per solve."""
    import numpy as np
    from synth import batched_systems
    systems = batched_systems()
    M = args.poles or 120
    kT = 0.01
    plan = nd.analyze_batched(systems, precision={"fp64": nd.NDSI_PREC_FP64, "split": nd.NDSI_PREC_SPLIT}[args.precision],
                              split_slices=args.slices)
    H = torch.as_tensor(np.concatenate([s.H for s in systems]), device="cuda")
    S = torch.as_tensor(np.concatenate([s.S for s in systems]), device="cuda")
    rho = torch.zeros(H.numel(), dtype=torch.float64, device="cuda")
    kts = np.full(len(systems), kT)
    ne = np.array([s.n_electrons for s in systems])
    ne_out = torch.zeros(len(systems), dtype=torch.float64, device="cuda")
    nd.ndsi_density_batched(plan, H, S, np.full(len(systems), MU), kts, M, rho, ne_out)   # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mu, n_e, rounds = nd.ndsi_find_mu_batched(plan, H, S, kts, M, ne, rho)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    line = {"metric": "chemical-potential search, all systems of the batched workload: batched sweeps per solve",
            "value": rounds, "unit": "sweeps", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "batched: 12 uneven systems (N 2048..32768), one plan", "poles": M, "kT": kT,
                       "precision": args.precision, "tolerance_electrons": 1e-8},
            "seconds": t, "mu": [float(v) for v in mu],
            "max_electron_error": float(np.max(np.abs(n_e - ne)))}
    print(json.dumps(line))
    return 0


def run_mu_search(args):
    """Chemical-potential search on the workload three ways: a bracket spanning the spectral
    bounds ("bounds"), no bracket (the paper's opening sequence with the retarded-Green-function
    trial mu, "dos_start") and the bracket proposed by the network trained here on exact-method mu
    of generated systems ("seeded"): contour sweeps and wall time per solve.  One JSON line; not
    part of the default run."""
    import numpy as np
    import torch
    from paper_1005_0088_gb300.build import build
    build()
    import paper_1005_0088_gb300 as nd
    from paper_1005_0088_gb300.mu_seed import MuSeed, build_dataset, features
    from synth import config_system, mu_training_systems, c5_family_systems
    torch.cuda.set_device(0)
    if args.config == "C4":
        return run_mu_search_batched(args, nd, torch)
    t0 = time.perf_counter()
    family = args.mu_family or ("c5" if args.config == "C5" else "generic")
    system = config_system(args.config)
    M_train = args.poles or system.meta["poles"]
    if family == "c5":
        X, T = build_dataset(c5_family_systems(args.mu_train, 1), n_poles=M_train)
    else:
        X, T = build_dataset(mu_training_systems(args.mu_train, 1))
    t_data = time.perf_counter() - t0
    model = MuSeed(seed=5)
    t0 = time.perf_counter()
    model.train(X, T, steps=3000, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    kT, M = system.meta["kT"], args.poles or system.meta["poles"]
    plan = nd.analyze_system(system, precision={"fp64": nd.NDSI_PREC_FP64, "split": nd.NDSI_PREC_SPLIT}[args.precision],
                             **_plan_options(args))
    H = torch.as_tensor(system.H, device="cuda")
    S = torch.as_tensor(system.S, device="cuda")
    rho = torch.zeros(system.nnz, dtype=torch.float64, device="cuda")
    ne = torch.zeros(1, dtype=torch.float64, device="cuda")
    nd.ndsi_density(plan, H, S, MU, kT, M, rho, ne)   # warm: tables, workspace, graph
    torch.cuda.synchronize()
    out = {}
    modes = ("dos_start", "seeded") if system.n > 20000 else ("bounds", "dos_start", "seeded")
    for mode in modes:
        t0 = time.perf_counter()
        lo = hi = 0.0
        if mode == "bounds":
            lo, hi = -1e6, 1e6      # clipped to the Gershgorin bounds of the pencil
        if mode == "seeded":
            lo, hi = model.bracket(features(plan, H, S, system.n_electrons, kT))
        mu, n_e, it = nd.ndsi_find_mu(plan, H, S, kT, M, system.n_electrons, rho, mu_lo=lo, mu_hi=hi)
        torch.cuda.synchronize()
        out[mode] = {"evaluations": it, "ms": (time.perf_counter() - t0) * 1e3, "mu": mu,
                     "electron_error": n_e - system.n_electrons}
    line = {"metric": "chemical-potential search: contour sweeps per solve",
            "value": out["seeded"]["evaluations"], "unit": "sweeps", "higher_is_better": False,
            "n_gpus": 1, "data": "synthetic",
            "config": {"workload": system.meta["label"], "poles": M, "kT": kT, "precision": args.precision,
                       "n_electrons": system.n_electrons, "tolerance_electrons": 1e-8},
            "bounds": out.get("bounds"), "dos_start": out["dos_start"], "seeded": out["seeded"],
            "seed_model": {"training_systems": args.mu_train, "family": family, "train_rmse_mu": model.rmse,
                           "dataset_s": t_data, "train_s": t_train,
                           "bracket_half_width": 3.0 * max(model.rmse or 0.05, 1e-3)}}
    print(json.dumps(line))
    return 0


def run_eigen(args):
    """Selected eigenstates near mu (App. B) on the workload: one factorisation at xi + i eta, the
    block shift-invert iteration to |Hc - eps Sc| < 1e-10, and the three-step solve timed alone
    (16 right-hand sides) against the HBM roofline of the fronts it reads.  One JSON line; not
    part of the default run."""
    import numpy as np
    import torch
    from paper_1005_0088_gb300.build import build
    build()
    import paper_1005_0088_gb300 as nd
    from synth import config_system
    torch.cuda.set_device(0)
    system = config_system(args.config)
    prec = {"fp64": nd.NDSI_PREC_FP64, "split": nd.NDSI_PREC_SPLIT}[args.precision]
    plan = nd.analyze_system(system, precision=prec, split_slices=args.slices)
    H = torch.as_tensor(system.H, device="cuda")
    S = torch.as_tensor(system.S, device="cuda")
    xi, n_states, block, eta = MU, 8, 12, 1e-3
    fp64_peak = nd.ndsi_fp64_peak()
    nd.ndsi_eigenstates(plan, H, S, xi, n_states, eta=eta, block=block)          # warm
    t0 = time.perf_counter()
    eps, C, res, iters = nd.ndsi_eigenstates(plan, H, S, xi, n_states, eta=eta, block=block)
    t_eig = time.perf_counter() - t0
    # the three-step solve alone, 16 right-hand sides, against the bytes of the fronts it reads
    f = nd.ndsi_factor_poles(plan, H, S, np.array([xi + 1j * eta]))
    k = 16
    Y = torch.randn(system.n, k, dtype=torch.complex128, device="cuda")
    X = torch.zeros_like(Y)
    for _ in range(3):
        nd.ndsi_factors_solve(f, 0, Y, X)
    reps = 10
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(reps):
        nd.ndsi_factors_solve(f, 0, Y, X)
    ev1.record()
    torch.cuda.synchronize()
    ms_solve = ev0.elapsed_time(ev1) / reps
    # algorithmic reads: A_J^{-1} (lower triangle) and L_RJ in the forward pass, L_RJ again in the
    # backward pass, once per 16 right-hand sides; plus the right-hand sides and solutions
    o = system.n // system.n_atoms
    s_sz = np.diff(nd.ndsi_plan_export(plan, "node_atoms")).astype(np.float64) * o
    r_sz = np.diff(nd.ndsi_plan_export(plan, "struct_ptr")).astype(np.float64) * o
    groups = (k + 7) // 8
    alg_bytes = groups * 16.0 * float(np.sum(s_sz * (s_sz + 1) / 2 + 2 * r_sz * s_sz)) + 4 * 16.0 * system.n * k
    # algorithmic flops: every complex term 8 flops, per right-hand side: A_J^{-1} y_J (s^2 terms,
    # each stored lower element used for two), L_RJ y_J and L_RJ^T x_R (r s terms each)
    alg_flops = 8.0 * k * float(np.sum(s_sz * s_sz + 2 * r_sz * s_sz))
    peak = _peaks().get("hbm_gbs", 6800.0)
    line = {"metric": "selected eigenstates near mu: wall time per solve", "value": t_eig * 1e3, "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": system.meta["label"], "n": system.n, "xi": xi, "eta": eta,
                       "n_states": n_states, "block": block, "precision": args.precision},
            "iterations": iters, "max_residual": float(np.max(res)), "eps": [float(e) for e in eps],
            "solve": {"rhs": k, "ms": ms_solve, "algorithmic_bytes": alg_bytes,
                      "gbs": alg_bytes / ms_solve / 1e6, "hbm_frac": alg_bytes / ms_solve / 1e6 / peak,
                      "roofline": {"bound": "alu", "unit": "TFLOP/s",
                                   "achieved": 0.75 * alg_flops / ms_solve / 1e9, "peak": fp64_peak,
                                   "frac": 0.75 * alg_flops / ms_solve / 1e9 / fp64_peak,
                                   "flop_count": "6 per complex term (the three-multiplication form "
                                                 "as executed; 8 in the conventional count)",
                                   "peak_source": "of measured (ndsi_fp64_peak in this run); the "
                                                  "solve is FP64-bound (each 16-byte factor element "
                                                  "feeds 3 real FMAs per right-hand side)"}}}
    if system.n <= 4096 and not args.no_cpu:
        from oracle.eigen import eigenstates_near
        Hd, Sd = system.dense()
        eps_ref, _ = eigenstates_near(Hd, Sd, xi, n_states)
        line["parity"] = {"max_abs_err_eps": float(np.max(np.abs(eps - eps_ref))), "oracle": "dense eigh"}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 10; 2 for the 3D metallic lattice, ~25 s a sweep, so "
                         "that the timed region stays near a minute)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ndsi", choices=["ndsi", "reference"])
    ap.add_argument("--config", default="C5", choices=["C1", "C2", "C3", "C4", "C5"])
    ap.add_argument("--precision", default="split", choices=["fp64", "split"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-parity", action="store_true", help="skip the sampled-column check")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every kernel directly instead of replaying a captured CUDA graph")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep every eligible GEMM of a split plan on the tensor cores")
    ap.add_argument("--energy", action="store_true",
                    help="each step also forms the energy density matrix (Eq. 10)")
    ap.add_argument("--by-level", action="store_true",
                    help="kernel breakdown of GEMM and slicing steps per tree level")
    ap.add_argument("--outer", type=int, default=0,
                    help="diagonal-block size of the two-level factorisation (0: library default)")
    ap.add_argument("--block", type=int, default=0,
                    help="FP64 pivot block size 16/32/64 (0: library default)")
    ap.add_argument("--bands", type=int, default=0,
                    help="TMEM accumulators of the split GEMM: 4 or 5 bands with a tail (0: one per "
                         "scale, the library default)")
    ap.add_argument("--slices", type=int, default=0,
                    help="BF16 slices per operand of the split path (4-7; 0: the library's choice)")
    ap.add_argument("--poles", type=int, default=0,
                    help="override the workload's pole count (small profiling runs only)")
    ap.add_argument("--fp64-poles", type=int, default=0,
                    help="poles of the FP64 comparison leg on systems above N = 20000 (0: 8)")
    ap.add_argument("--lattice", default="",
                    help="profiling workload NXxNYxNZxO (3D cubic, kT 0.01, 40 poles) instead of --config")
    ap.add_argument("--leaf", type=int, default=0,
                    help="innermost-domain size of the dissection in atoms (0: library default)")
    ap.add_argument("--far-ratio", type=float, default=0.0,
                    help="split plans: poles with z_p >= ratio z_1 use one slice fewer (0: library "
                         "default, negative: off)")
    ap.add_argument("--no-other", action="store_true",
                    help="skip the run of the other precision (split-vs-FP64 speedup)")
    ap.add_argument("--mu-search", action="store_true",
                    help="time the chemical-potential search, plain and seeded by the trained network")
    ap.add_argument("--eigen", action="store_true",
                    help="time the selected-eigenstates solver (App. B) near mu")
    ap.add_argument("--mu-train", type=int, default=2000,
                    help="generated systems the mu-search network is trained on")
    ap.add_argument("--mu-family", default="", choices=["", "generic", "c5"],
                    help="training systems: small varied lattices, or the 3D metallic recipe's "
                         "family (default: c5 for --config C5)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 2 if args.config == "C5" and not (args.poles or args.lattice) else 10
    if args.impl == "reference":
        return run_reference(args)
    if args.mu_search:
        return run_mu_search(args)
    if args.eigen:
        return run_eigen(args)
    return run_ndsi(args)


if __name__ == "__main__":
    sys.exit(main())
