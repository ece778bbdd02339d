#!/usr/bin/env python
"""Benchmark: poles x N per second of the selected-inversion density path on one GB300.

Step = one density evaluation rho(mu) (assembly, factor, selected inversion and the residue sum
for every pole of the workload), inputs resident in HBM.  Default workload: the 2D square sheet
of 32 x 32 atoms x 4 orbitals (N = 4096), 80 poles, kT = 0.01 Ha, FP64 path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ndsi|reference] [--config C2]

Under torchrun every rank runs its own replica of the workload (weak scaling, no data-path
collective); the max step time over ranks is reported.  `--impl reference` times the CPU
oracle (dense generalized eigendecomposition + the same pole-truncated Fermi function) on the
same workload, on rank 0 only.
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

METRIC = "poles x N per second (selected inversion); split-prec vs FP64 speedup at 1e-9"
UNIT = "poles*N/s"
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 (DFMA) rate from the hardware table
MU = -0.12


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _max_over_ranks(x, dist, world, device):
    """Largest value of x over all ranks (the slowest replica sets the job's time)."""
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
    """Whole-job throughput: every replica processes units_per_rank per step."""
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
        sms, mx, reasons = [], 0.0, set()
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
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": mx or None, "reasons": sorted(reasons), "samples": len(sms)}


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


def cpu_single_core_rate(config, mu):
    """The oracle's route 1 on one host core (a child process with every BLAS pool at one thread):
    poles x N per second, or None when the child fails."""
    import subprocess
    code = ("import time, json; from synth import config_system; "
            "from oracle.dense import generalized_eig, density_eig, on_pattern; "
            f"s = config_system({config!r}); Hd, Sd = s.dense(); kT, M = s.meta['kT'], s.meta['poles']; "
            "ts = []\n"
            "for _ in range(3):\n"
            "    t0 = time.perf_counter(); e, C = generalized_eig(Hd, Sd); "
            f"on_pattern(density_eig(e, C, {mu!r}, kT, M), s); ts.append(time.perf_counter() - t0)\n"
            "print(json.dumps(M * s.n / min(ts)))")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                             text=True, timeout=300)
        return float(out.stdout.strip().splitlines()[-1]) if out.returncode == 0 else None
    except (subprocess.SubprocessError, ValueError, IndexError):
        return None


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
    from synth import config_system
    from oracle.dense import generalized_eig, density_eig, on_pattern
    system = config_system(args.config)
    kT, M = system.meta["kT"], system.meta["poles"]
    Hd, Sd = system.dense()
    def step():
        eps, C = generalized_eig(Hd, Sd)
        on_pattern(density_eig(eps, C, MU, kT, M), system)
    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = M * system.n / t
    cores = os.cpu_count()
    sample = (f"one full density evaluation of {args.config} per step by the oracle's dense "
              f"generalized eigendecomposition (N={system.n}) and the {M}-pole Fermi sum")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": system.meta["label"], "n": system.n, "poles": M, "kT": kT,
                       "mu": MU},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _kernel_totals(prof):
    """Aggregate per-step profiler entries ("gemm_split:schur") into kernels ("gemm_split")."""
    out = {}
    for name, v in prof.items():
        k = name.split(":")[0]
        o = out.setdefault(k, dict(launches=0, ms=0.0, flops=0.0, bytes=0.0, tensor_flops=0.0))
        for f in o:
            o[f] += v[f]
    return out


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, averaged over the kernel's
# launches in one timed sweep) from an ncu capture of the same build and workload with default
# options.  Entries are removed whenever the kernel changes.
TRAFFIC_PER_LAUNCH = {("C2", "fp64", "gemm_f64"): 55.06e6}


def _roofline(prof, steps, peaks, traffic_key=None):
    kern = _kernel_totals(prof)
    dname, d = max(kern.items(), key=lambda kv: kv[1]["ms"])
    total = sum(v["ms"] for v in kern.values())
    if dname == "gemm_split":
        peak = peaks.get("bf16_tflops_sustained", 1738.1)
        achieved = d["tensor_flops"] / (d["ms"] * 1e-3) / 1e12
        r = {"bound": "tensor", "unit": "TFLOP/s", "peak": peak,
             "peak_source": "of measured (MEASURED_PEAKS.json bf16_tflops_sustained; the kernel runs "
                            "inside a long step)",
             "fp64_equivalent_tflops": d["flops"] / (d["ms"] * 1e-3) / 1e12}
    elif dname in ("gemm_f64", "diaginv"):
        peak = FP64_PEAK_TFLOPS
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
        r = {"bound": "alu", "unit": "TFLOP/s", "peak": peak,
             "peak_source": "nominal GB300 FP64 DFMA rate from the hardware table (1.25 TFLOP/s); "
                            "a DFMA loop measured 1.01 TFLOP/s"}
    else:
        peak = peaks.get("hbm_gbs", 6800.0)
        achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
        r = {"bound": "hbm", "unit": "GB/s", "peak": peak,
             "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)"}
    traffic = TRAFFIC_PER_LAUNCH.get(traffic_key + (dname,)) if traffic_key else None
    r.update({"kernel": dname, "achieved": achieved, "frac": achieved / peak, "traffic": traffic,
              "launches": d["launches"], "kernel_ms_per_step": d["ms"] / steps,
              "share": d["ms"] / total})
    return r, kern


def _autotune(nd, args, plan, H, S, kT, M):
    """Per-step tensor-core / FP64 choice of a split plan, made once before any timing."""
    if args.no_autotune:
        return None
    n_split, n_fp64 = nd.ndsi_autotune(plan, H, S, MU, kT, M)
    return {"tensor_core_steps": n_split, "fp64_steps": n_fp64}


def _measure(nd, torch, plan, H, S, rho, ne, kT, M, steps, warmup, stream, flush, by_level=False,
             e=None):
    """Time `steps` density sweeps as the library runs them (one captured CUDA graph per sweep),
    then repeat them with direct launches and per-launch CUDA events for the kernel breakdown.
    With `e` (an nnz device buffer) each sweep also forms the energy density matrix."""
    def step():
        if e is None:
            nd.ndsi_density(plan, H, S, MU, kT, M, rho, ne, stream=stream)
        else:
            nd.ndsi_density_energy(plan, H, S, MU, kT, M, rho, e, ne, stream=stream)

    def timed_steps(ahead):
        # L2 flush, start event, sweep, end event per step, all on the launch stream; with
        # `ahead` the steps are enqueued back to back (the host runs ahead of the GPU, so host
        # scheduling noise does not open gaps between the events), else synchronised per step
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
    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    # the timed region alone is what `ncu --profile-from-start off` records (a no-op otherwise)
    torch.cuda.profiler.start()
    times = timed_steps(True)
    torch.cuda.profiler.stop()
    nd.ndsi_profile_enable(plan, True, by_level=by_level)
    prof_times = timed_steps(False)
    prof = nd.ndsi_profile_read(plan)
    nd.ndsi_profile_enable(plan, False)
    return times, prof, prof_times


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
    system = config_system(args.config)
    kT, M = system.meta["kT"], system.meta["poles"]
    if args.poles:
        M = args.poles
    plan = nd.analyze_system(system, precision=prec_code[args.precision], split_slices=args.slices,
                             outer_block=args.outer, block=args.block, split_bands=args.bands)
    info = nd.ndsi_plan_info(plan)
    dev = torch.device("cuda", local)
    H = torch.as_tensor(system.H, device=dev)
    S = torch.as_tensor(system.S, device=dev)
    tune = _autotune(nd, args, plan, H, S, kT, M)
    if args.no_graph:
        nd.ndsi_graph_enable(plan, False)
    rho = torch.zeros(system.nnz, dtype=torch.float64, device=dev)
    ne = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()

    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        e_buf = torch.zeros_like(rho) if args.energy else None
        times, prof, prof_times = _measure(nd, torch, plan, H, S, rho, ne, kT, M, args.steps,
                                           args.warmup, stream, flush, by_level=args.by_level, e=e_buf)
        graph_nodes = nd.ndsi_graph_info(plan)
    if world > 1:
        dist.barrier()
    total_ms = _max_over_ranks(sum(times), dist, world, dev)
    ms_step = total_ms / args.steps
    value = _job_value(M * system.n, world, ms_step)
    rho_main = rho.cpu().numpy()
    # end to end through the public API with pinned host buffers (copies inside the call)
    Hh = torch.as_tensor(system.H).pin_memory()
    Sh = torch.as_tensor(system.S).pin_memory()
    rho_h = torch.zeros(system.nnz, dtype=torch.float64).pin_memory()
    ne_h = torch.zeros(1, dtype=torch.float64).pin_memory()
    nd.ndsi_density(plan, Hh, Sh, MU, kT, M, rho_h, ne_h, stream=stream)
    e2e_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nd.ndsi_density(plan, Hh, Sh, MU, kT, M, rho_h, ne_h, stream=stream)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = _max_over_ranks(sum(e2e_times) / len(e2e_times), dist, world, dev)
    # the other precision on the same workload: split-vs-FP64 speedup and rho difference
    other = None
    if not args.no_other and rank == 0:
        oprec = "split" if args.precision == "fp64" else "fp64"
        plan2 = nd.analyze_system(system, precision=prec_code[oprec], split_slices=args.slices,
                                  outer_block=args.outer, block=args.block, split_bands=args.bands)
        tune2 = _autotune(nd, args, plan2, H, S, kT, M)
        rho2 = torch.zeros_like(rho)
        ne2 = torch.zeros_like(ne)
        t2, prof2, _ = _measure(nd, torch, plan2, H, S, rho2, ne2, kT, M, args.steps, args.warmup,
                                stream, flush)
        ms2 = sum(t2) / len(t2)
        ms_split, ms_fp64 = (ms2, ms_step) if oprec == "split" else (ms_step, ms2)
        rl2, k2 = _roofline(prof2, args.steps, _peaks())
        other = {"precision": oprec, "ms_per_step": ms2, "value": M * system.n / (ms2 * 1e-3),
                 "split_speedup_vs_fp64": ms_fp64 / ms_split, "autotune": tune2,
                 "abs_n_elec_diff_vs_headline": abs(float(ne2.cpu()[0]) - float(ne.cpu()[0])),
                 "max_abs_rho_diff_vs_headline": float(np.max(np.abs(rho2.cpu().numpy() - rho_main))),
                 "roofline": rl2,
                 "kernels": {k: {"launches": v["launches"] // args.steps, "ms_per_step": v["ms"] / args.steps}
                             for k, v in k2.items()}}
        del plan2
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    default_opts = not (args.poles or args.outer or args.block or args.slices or args.bands)
    roofline, kern = _roofline(prof, args.steps, _peaks(),
                               (args.config, args.precision) if default_opts else None)
    launches = sum(v["launches"] for v in kern.values())
    # parity spot check outside the timed region: sampled columns from the oracle
    parity = None
    if not args.no_parity:
        from oracle.dense import density_columns
        rng = np.random.default_rng(11)
        cols = sorted(rng.choice(system.n, 3, replace=False).tolist())
        ref = density_columns(system, MU, kT, M, cols)
        rows = system.rows()
        err = 0.0
        for t_, j in enumerate(cols):
            sel = np.nonzero(system.col == j)[0]
            err = max(err, float(np.max(np.abs(rho_main[sel] - ref[rows[sel], t_]))))
        parity = {"max_abs_err_rho": err, "columns": cols,
                  "tolerance": 1e-10 if args.precision == "fp64" else 1e-9}
        if e_buf is not None:
            from oracle.dense import energy_density_columns
            e_main = e_buf.cpu().numpy()
            eref = energy_density_columns(system, MU, kT, M, cols)
            ee = 0.0
            for t_, j in enumerate(cols):
                sel = np.nonzero(system.col == j)[0]
                ee = max(ee, float(np.max(np.abs(e_main[sel] - eref[rows[sel], t_]))))
            parity["max_abs_err_energy_density"] = ee
    cpu = None
    ne_gpu = float(ne.cpu()[0])
    n_elec = {"value": ne_gpu}
    golden = os.path.join(ROOT, "tests", "golden", "c3_electron_count.txt")
    if args.config == "C3" and M == 80 and os.path.exists(golden):
        # the oracle's count for this workload (eigenvalues by LAPACK, stored by
        # tests/golden/make_c3_electron_count.py): too slow to recompute inside the bench
        with open(golden) as fh:
            ne_ref = float([ln for ln in fh if ln.strip() and not ln.startswith("#")][0])
        n_elec.update(oracle=ne_ref, abs_err=abs(ne_gpu - ne_ref), oracle_source="stored (oracle eigenvalues)")
    if world == 1 and not args.no_cpu:
        v, reps, t_rep, ne_oracle = cpu_oracle_rate(system, MU, kT, M)
        n_elec.update(oracle=ne_oracle, abs_err=abs(ne_gpu - ne_oracle))
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{reps} full density evaluations of the workload by dense generalized "
                         f"eigendecomposition + {M}-pole Fermi sum ({t_rep:.2f} s each)"}
        extra = {}
        if system.n <= 1024:
            v1 = cpu_single_core_rate(args.config, MU)
            if v1 is not None:
                extra["oracle_one_core"] = {"value": v1, "unit": UNIT, "cores": 1}
        if system.n <= 16384:
            vs, npl, tpl = cpu_sparse_lu_rate(system, MU, kT, M)
            extra["scipy_sparse_lu"] = {"value": vs, "unit": UNIT, "cores": os.cpu_count(),
                                        "sample": f"SuperLU factorisation of {npl} poles, "
                                                  f"{tpl * 1e3:.1f} ms each, scaled to {M + 1} "
                                                  "points; factorisation only (no selected "
                                                  "inversion), a lower bound of a CPU sparse route"}
        if extra:
            cpu["other_cpu_routes"] = extra
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else f"bf16x{info['split_slices']}->f64",
            "data": "synthetic",
            "config": {"workload": system.meta["label"] + f", {M} poles, {args.precision} path"
                                   + (", rho and energy density matrix" if args.energy else ""),
                       "n": system.n, "poles": M, "kT": kT, "mu": MU, "nnz": system.nnz,
                       "precision": args.precision, "split_slices": info["split_slices"],
                       "split_bands": info["split_bands"],
                       "l2": "flushed (256 MB write) before every timed step",
                       "flops_per_pole": info["flops_per_pole"], "parallelism": f"replicas x{world}"},
            "e2e": {"value": world * M * system.n / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": 2 * 8 * system.nnz,
                    "d2h_bytes_per_step": 8 * system.nnz + 8},
            "gpu_launches": launches,
            "step_ms": [round(t, 4) for t in times],
            "autotune": tune,
            "graph": {"kernel_nodes": graph_nodes,
                      "ms_per_step_direct_launches": sum(prof_times) / len(prof_times),
                      "note": "timed steps replay one captured CUDA graph per sweep; the kernel "
                              "breakdown and roofline come from the same steps repeated with direct "
                              "launches bracketed by CUDA events on the launch stream"},
            "roofline": roofline, "clocks": clk.summary(), "cpu_baseline": cpu,
            "parity": parity, "n_elec": n_elec, "other_precision": other,
            "kernels": {k: {"launches": v["launches"] // args.steps, "ms_per_step": v["ms"] / args.steps,
                            "gbs": v["bytes"] / max(v["ms"], 1e-9) / 1e6,
                            "tflops": v["flops"] / max(v["ms"], 1e-9) / 1e9}
                        for k, v in kern.items()},
            "steps_detail": {k: {"launches": v["launches"] // args.steps, "ms_per_step": v["ms"] / args.steps}
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
    plan = nd.analyze_batched(systems, precision=prec_code[args.precision], split_slices=args.slices,
                              outer_block=args.outer, block=args.block, split_bands=args.bands)
    info = nd.ndsi_plan_info(plan)
    dev = torch.device("cuda", local)
    H = torch.as_tensor(np.concatenate([s.H for s in systems]), device=dev)
    S = torch.as_tensor(np.concatenate([s.S for s in systems]), device=dev)
    nnz = int(H.shape[0])
    rho = torch.zeros(nnz, dtype=torch.float64, device=dev)
    ne = torch.zeros(len(systems), dtype=torch.float64, device=dev)
    mus = np.full(len(systems), MU)
    kts = np.full(len(systems), kT)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        nd.ndsi_density_batched(plan, H, S, mus, kts, M, rho, ne, stream=stream)
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
    nd.ndsi_density_batched(plan, Hh, Sh, mus, kts, M, rho_h, ne_h, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nd.ndsi_density_batched(plan, Hh, Sh, mus, kts, M, rho_h, ne_h, stream=stream)
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
    roofline, kern = _roofline(prof, args.steps, _peaks())
    line = {"metric": METRIC, "value": _job_value(M * ntot, world, ms), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else f"bf16x{info['split_slices']}->f64", "data": "synthetic",
            "config": {"workload": f"batched: {M} poles x {len(systems)} uneven systems "
                                   f"(N {min(s.n for s in systems)}..{max(s.n for s in systems)}), "
                                   f"{args.precision} path, one launch per tree level",
                       "n_total": ntot, "poles": M, "kT": kT, "nnz": nnz, "precision": args.precision,
                       "flops_per_pole": info["flops_per_pole"], "n_levels": info["n_levels"],
                       "l2": "flushed (256 MB write) before every timed step"},
            "e2e": {"value": _job_value(M * ntot, world, e2e_s * 1e3), "unit": UNIT,
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
    from synth import config_system, mu_training_systems
    torch.cuda.set_device(0)
    if args.config == "C4":
        return run_mu_search_batched(args, nd, torch)
    t0 = time.perf_counter()
    X, T = build_dataset(mu_training_systems(args.mu_train, 1))
    t_data = time.perf_counter() - t0
    model = MuSeed(seed=5)
    t0 = time.perf_counter()
    model.train(X, T, steps=3000, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    system = config_system(args.config)
    kT, M = system.meta["kT"], args.poles or system.meta["poles"]
    plan = nd.analyze_system(system, precision={"fp64": nd.NDSI_PREC_FP64, "split": nd.NDSI_PREC_SPLIT}[args.precision],
                             split_slices=args.slices)
    H = torch.as_tensor(system.H, device="cuda")
    S = torch.as_tensor(system.S, device="cuda")
    rho = torch.zeros(system.nnz, dtype=torch.float64, device="cuda")
    ne = torch.zeros(1, dtype=torch.float64, device="cuda")
    nd.ndsi_density(plan, H, S, MU, kT, M, rho, ne)   # warm: tables, workspace, graph
    torch.cuda.synchronize()
    out = {}
    for mode in ("bounds", "dos_start", "seeded"):
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
            "bounds": out["bounds"], "dos_start": out["dos_start"], "seeded": out["seeded"],
            "seed_model": {"training_systems": args.mu_train, "train_rmse_mu": model.rmse,
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
                      "roofline": {"bound": "alu", "unit": "TFLOP/s", "achieved": alg_flops / ms_solve / 1e9,
                                   "peak": 1.25, "frac": alg_flops / ms_solve / 1e9 / 1.25,
                                   "peak_source": "nominal GB300 FP64 DFMA rate (1.25 TFLOP/s); the "
                                                  "solve is FP64-bound (each 16-byte factor element "
                                                  "feeds 3 real FMAs per right-hand side: the "
                                                  "three-multiplication form executes 6 of the 8 "
                                                  "counted flops)"}}}
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
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ndsi", choices=["ndsi", "reference"])
    ap.add_argument("--config", default="C2", choices=["C1", "C2", "C3", "C4", "C5"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "split"])
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
                    help="TMEM accumulator bands of the split GEMM, 4 or 5 (0: the library's choice)")
    ap.add_argument("--slices", type=int, default=0,
                    help="BF16 slices per operand of the split path (4-7; 0: the library's choice)")
    ap.add_argument("--poles", type=int, default=0,
                    help="override the workload's pole count (small profiling runs only)")
    ap.add_argument("--no-other", action="store_true",
                    help="skip the run of the other precision (split-vs-FP64 speedup)")
    ap.add_argument("--mu-search", action="store_true",
                    help="time the chemical-potential search, plain and seeded by the trained network")
    ap.add_argument("--eigen", action="store_true",
                    help="time the selected-eigenstates solver (App. B) near mu")
    ap.add_argument("--mu-train", type=int, default=2000,
                    help="generated systems the mu-search network is trained on")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mu_search:
        return run_mu_search(args)
    if args.eigen:
        return run_eigen(args)
    return run_ndsi(args)


if __name__ == "__main__":
    sys.exit(main())
