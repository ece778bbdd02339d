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
    """Time the oracle's route 1 (dense eigendecomposition + truncated Fermi sum on the pattern)."""
    from oracle.dense import generalized_eig, density_eig, on_pattern
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
    return M * system.n / t, len(times), t


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

    system = config_system(args.config)
    kT, M = system.meta["kT"], system.meta["poles"]
    prec = {"fp64": nd.NDSI_PREC_FP64, "split": nd.NDSI_PREC_SPLIT}[args.precision]
    plan = nd.analyze_system(system, precision=prec)
    info = nd.ndsi_plan_info(plan)
    dev = torch.device("cuda", local)
    H = torch.as_tensor(system.H, device=dev)
    S = torch.as_tensor(system.S, device=dev)
    rho = torch.zeros(system.nnz, dtype=torch.float64, device=dev)
    ne = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def step():
        nd.ndsi_density(plan, H, S, MU, kT, M, rho, ne, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    nd.ndsi_profile_enable(plan, True)
    times = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    prof = nd.ndsi_profile_read(plan)
    nd.ndsi_profile_enable(plan, False)
    total_ms = sum(times)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / args.steps
    value = world * M * system.n / (ms_step * 1e-3)
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
    e2e_s = sum(e2e_times) / len(e2e_times)
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    if rank != 0:
        dist.destroy_process_group() if world > 1 else None
        return 0
    # roofline of the dominant kernel family
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    dname, d = dom
    peaks = _peaks()
    if dname.startswith("gemm_f64") or dname == "diaginv":
        bound, unit, peak = "alu", "TFLOP/s", FP64_PEAK_TFLOPS
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
        peak_note = "nominal GB300 FP64 DFMA rate (hardware table); measured DFMA loop: 1.01 TFLOP/s"
    else:
        bound, unit = "hbm", "GB/s"
        peak = peaks.get("hbm_gbs", 6800.0)
        achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
        peak_note = "of measured (MEASURED_PEAKS.json hbm_gbs)"
    roofline = {"kernel": dname, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": None, "peak_source": peak_note,
                "launches": d["launches"], "kernel_ms_per_step": d["ms"] / args.steps,
                "share": d["ms"] / sum(v["ms"] for v in prof.values())}
    launches = sum(v["launches"] for v in prof.values()) // args.steps
    # parity spot check outside the timed region: sampled columns from the oracle
    parity = None
    if not args.no_parity:
        from oracle.dense import density_columns
        rho_np = rho.cpu().numpy()
        rng = np.random.default_rng(11)
        cols = sorted(rng.choice(system.n, 3, replace=False).tolist())
        ref = density_columns(system, MU, kT, M, cols)
        rows = system.rows()
        err = 0.0
        for t_, j in enumerate(cols):
            sel = np.nonzero(system.col == j)[0]
            err = max(err, float(np.max(np.abs(rho_np[sel] - ref[rows[sel], t_]))))
        parity = {"max_abs_err_rho": err, "columns": cols, "tolerance": 1e-10}
    cpu = None
    if world == 1 and not args.no_cpu:
        v, reps, t_rep = cpu_oracle_rate(system, MU, kT, M)
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{reps} full density evaluations of the workload by dense generalized "
                         f"eigendecomposition + {M}-pole Fermi sum ({t_rep:.2f} s each)"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "bf16x{}->f64".format(6),
            "data": "synthetic",
            "config": {"workload": system.meta["label"] + f", {M} poles, {args.precision} path",
                       "n": system.n, "poles": M, "kT": kT, "mu": MU, "nnz": system.nnz,
                       "precision": args.precision, "l2": "flushed (256 MB write) before every timed step",
                       "flops_per_pole": info["flops_per_pole"], "parallelism": f"replicas x{world}"},
            "e2e": {"value": world * M * system.n / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": 2 * 8 * system.nnz,
                    "d2h_bytes_per_step": 8 * system.nnz + 8},
            "gpu_launches": launches * args.steps,
            "roofline": roofline, "clocks": clk.summary(), "cpu_baseline": cpu,
            "parity": parity,
            "kernels": {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps}
                        for k, v in prof.items()}}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ndsi", choices=["ndsi", "reference"])
    ap.add_argument("--config", default="C2", choices=["C1", "C2", "C3"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "split"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-parity", action="store_true", help="skip the sampled-column check")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ndsi(args)


if __name__ == "__main__":
    sys.exit(main())
