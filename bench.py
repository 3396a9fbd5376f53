#!/usr/bin/env python
"""Throughput of the MGRIT solve of the 2-D Riesz SFDE on GB300: space-time DOF-updates/s.

One "step" is one complete MGRIT solve (all V-cycles to the stopping tolerance) of the
workload ``sine_N255_Nt1024``: N_x = N_y = 255, N_t = 1024 uniform steps on (0,1]^3,
beta = 0.6, gamma = 0.9, K_x = 1, K_y = 0.5, sixteen seeded sine modes for psi_0, f = 0,
V-cycle with m = 8.  value = N_x N_y N_t / (device seconds per solve), summed over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--precision ...]

--impl reference times the FP64 CPU oracle (the slow, plain implementation that the tests
compare against) on the host cores; it never touches the GPU.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from sfde_workloads import WORKLOADS  # noqa: E402

METRIC = "space-time DOF-updates/s to 1e-8 rel. residual: mixed/batched vs FP64 MGRIT, 1 GB300"
UNIT = "DOF-updates/s"
WORKLOAD = "sine_N255_Nt1024"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Nominal GB300 rates (TFLOP/s): FP64 and BF16 dense; FP64 peak = measured BF16 x nominal ratio.
NOMINAL_FP64_TFLOPS = 1.25
NOMINAL_BF16_TFLOPS = 2250.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    try:
        p = json.load(open(PEAKS_FILE))
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = {
    "k_slice_gemm_fp64": ("step_fp64.cu",),
    "k_tc_slice_gemm": ("gemm_tc.cu", "tc_common.cuh"),
    "k_fused_step": ("fused_step.cu", "tc_common.cuh"),
    "k_digit_gemm_int": ("ozaki.cu", "tc_common.cuh"),
    "k_split_pair+k_combine_int": ("resid_int.cu",),
}


def kernel_source_sha(kernel: str):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, ()):
        h.update(open(os.path.join(ROOT, "paper_1805_06688_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel: str, flops_per_launch: float, bytes_per_launch: float):
    """DRAM bytes per launch from a committed ncu summary (profiles/traffic.json), scaled by the
    algorithmic work of the launch (flops, or bytes for a kernel without flops), if the counters
    were taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))[kernel]
    except Exception:
        return None
    if d.get("source_sha") != kernel_source_sha(kernel):
        return None
    if "dram_bytes_per_flop" in d:
        return d["dram_bytes_per_flop"] * flops_per_launch
    return d["dram_bytes_per_alg_byte"] * bytes_per_launch


# ----------------------------------------------------------------------------- oracle timing

def oracle_rate(w, iters_needed: int, coarse: str, budget_s: float = 20.0):
    """FP64 CPU oracle on a bounded sample: one V-cycle of the nodal Algorithm 1 (all levels),
    extrapolated to the V-cycles the full solve needs.  Returns (rate, seconds, cores, sample)."""
    from oracle import mgrit as omgrit, sfde as osfde
    t = w.t()
    prob = osfde.SFDE(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t)
    prob.eig()
    psi = w.initial()
    t0 = time.perf_counter()
    r = omgrit.mgrit(prob, psi, w.forcing(), m=w.m, max_levels=w.max_levels, coarse=coarse,
                     rel_tol=0.0, max_iter=1)
    dt = time.perf_counter() - t0
    rate = w.space_time_updates / (dt * iters_needed)
    sample = (f"one V-cycle ({r.step_solves} step solves, all {r.levels} levels) of the oracle's nodal "
              f"FP64 MGRIT on {w.name}, extrapolated to the {iters_needed} V-cycles of the full solve")
    return rate, dt, os.cpu_count(), sample


def oracle_iterations(w, coarse: str) -> int:
    from oracle import mgrit as omgrit, sfde as osfde
    prob = osfde.SFDE(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, w.t())
    r = omgrit.mgrit_modal(prob, w.initial(), w.forcing(), m=w.m, max_levels=w.max_levels,
                           coarse=coarse, rel_tol=w.rel_tol, max_iter=400)
    return r.iters


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    coarse = "be"  # the coarse propagator the solver picks for this workload (bound of Thm 3.1 > 1)
    iters = oracle_iterations(w, coarse)
    rates, secs = [], []
    for k in range(args.warmup + args.steps):
        rate, dt, cores, sample = oracle_rate(w, iters, coarse)
        if k >= args.warmup:
            rates.append(rate)
            secs.append(dt * iters)
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "nt": w.nt, "m": w.m,
                   "rel_tol": w.rel_tol, "coarse": coarse, "solver": "FP64 CPU oracle, Algorithm 1"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- roofline

KERNEL_CLASSES = (  # the library's accounting classes (include/sfde.h, sfde_profile)
    ("k_slice_gemm_fp64", "FP64 slice GEMM of a step", "alu"),
    ("k_slice_gemm_fp64", "FP64 slice GEMM of the space-time residual", "alu"),
    ("k_tc_slice_gemm", "tcgen05 slice GEMM of a low-precision step (BF16/TF32)", "tc"),
    ("k_fused_step", "fused BF16 spectral step: four tcgen05 products per slice on chip", "tc"),
    ("k_digit_gemm_int", "digit-split residual products: up to 28 BF16 tcgen05 products, exact int64", "tc"),
    ("k_split_pair+k_combine_int", "integer residual assembly (exponents, digits, combination)", "hbm"),
)


def roofline_from_profile(prof, precision: str):
    """Roofline of the kernel class with the largest device time, plus a per-class breakdown.

    Each class's launches are timed with CUDA events inside the solve (a long step), so the
    denominators are the sustained measured rates.  FP64 SIMT GEMMs are bound by the FP64 pipe
    (measured BF16 x nominal FP64/BF16); tensor-core kernels are placed by algorithmic intensity
    against the ridge point (below it: HBM bandwidth, above it: the tensor pipe of their dtype);
    the integer assembly kernels move bytes only."""
    pk, src = peaks()
    bf16 = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    fp64_peak = bf16 * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS
    kernels = []
    for k, (name, what, kind) in enumerate(KERNEL_CLASSES):
        if k >= len(prof.launches):
            break
        n, ms, fl, by = prof.launches[k], prof.ms[k], prof.flops[k], prof.bytes[k]
        if n == 0 or ms <= 0:
            continue
        tfs = fl / (ms * 1e-3) / 1e12
        gbs = by / (ms * 1e-3) / 1e9
        tc_peak = bf16 * (0.5 if (k == 2 and precision == "mixed-tf32") else 1.0)
        if kind == "alu":
            bound, ach, peak, unit = "alu", tfs, fp64_peak, "TFLOP/s"
            psrc = f"{src} sustained BF16 {bf16} TFLOP/s x nominal FP64/BF16 {NOMINAL_FP64_TFLOPS}/{NOMINAL_BF16_TFLOPS}"
        elif kind == "hbm" or fl / by < tc_peak * 1e12 / (pk["hbm_gbs"] * 1e9):
            bound, ach, peak, unit = "hbm", gbs, pk["hbm_gbs"], "GB/s"
            psrc = f"{src} HBM copy bandwidth"
        else:
            bound, ach, peak, unit = "tensor", tfs, tc_peak, "TFLOP/s"
            psrc = f"{src} sustained BF16 dense" + (" x 1/2 (TF32 nominal ratio)" if tc_peak < bf16 else "")
        kernels.append({
            "kernel": name, "what": what, "launches": int(n), "ms": ms, "share": None,
            "bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
            "peak_source": psrc, "avg_launch_us": 1e3 * ms / n,
            "algorithmic_flops_per_launch": fl / n, "algorithmic_bytes_per_launch": by / n,
            "tflops": tfs, "gbs": gbs,
        })
    tot = sum(k["ms"] for k in kernels) or 1.0
    for k in kernels:
        k["share"] = k["ms"] / tot
    dom = max(kernels, key=lambda k: k["ms"])
    roofline = {
        "bound": dom["bound"], "achieved": dom["achieved"], "peak": dom["peak"], "unit": dom["unit"],
        "frac": dom["frac"],
        "traffic": traffic_from_profile(dom["kernel"], dom["algorithmic_flops_per_launch"],
                                        dom["algorithmic_bytes_per_launch"]),
        "kernel": f"{dom['kernel']} ({dom['what']})", "peak_source": dom["peak_source"],
        "launches": dom["launches"], "avg_launch_us": dom["avg_launch_us"],
        "algorithmic_flops_per_launch": dom["algorithmic_flops_per_launch"],
        "algorithmic_bytes_per_launch": dom["algorithmic_bytes_per_launch"],
        "share_of_accounted_time": dom["share"],
    }
    return roofline, kernels


# ----------------------------------------------------------------------------- ranks

def whole_job_rate(seconds_local: float, units_local: float, world: int, device=None):
    """Whole-job throughput over `world` ranks: the units all ranks processed over the slowest
    rank's time (max over ranks, one all-reduce each; `device` holds the reduction tensors: the
    rank's GPU under NCCL, the CPU under gloo).  Returns (units per second, max seconds)."""
    if world <= 1:
        return units_local / seconds_local, seconds_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


# ----------------------------------------------------------------------------- GPU arm

def run_ours(args, w):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_1805_06688_gb300 as sfde
    if not os.path.exists(sfde.library_path):
        from paper_1805_06688_gb300.build import build
        build()

    stream = torch.cuda.current_stream(dev)
    prec = {"fp64": sfde.PREC_FP64, "mixed-bf16": sfde.PREC_MIXED_BF16,
            "mixed-tf32": sfde.PREC_MIXED_TF32, "mixed-auto": sfde.PREC_MIXED_AUTO}[args.precision]
    t = w.t()
    psi = w.initial()
    P = sfde.Problem(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t, w.omega, precision=prec,
                     stream=stream.cuda_stream)
    P.set_initial(torch.from_numpy(psi).to(dev))
    P.set_forcing(w.forcing())
    # FP64: C-point residual to the workload's tolerance; mixed: FP64 space-time residual to 1e-8
    # relative (max-norm error against the exact solution ~1e-10, checked by the GPU tests)
    tol = w.rel_tol if prec == sfde.PREC_FP64 else 1e-8
    kw = dict(m=w.m, max_levels=w.max_levels, coarse=sfde.COARSE_AUTO, rel_tol=tol, max_iter=400)
    UT = torch.zeros((w.ny, w.nx), dtype=torch.float64, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    stats = None
    for _ in range(args.warmup):
        _, stats = P.mgrit(U_T=UT, **kw)
    # timed region: inputs (the 1025-slice FP64 space-time iterate, 537 MB) exceed L2
    P.profile_enable(False)
    barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            _, stats = P.mgrit(U_T=UT, **kw)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    launches = P.profile_read().kernel_launches
    value, sec = whole_job_rate(ev0.elapsed_time(ev1) * 1e-3 / args.steps, w.space_time_updates, world, dev)
    ms = 1e3 * sec

    # dominant kernel: per-launch CUDA-event durations over one more solve
    P.profile_enable(True)
    P.mgrit(U_T=UT, **kw)
    prof = P.profile_read()
    P.profile_enable(False)
    roofline, kernels = roofline_from_profile(prof, args.precision)

    # end to end through the C ABI with host buffers: psi_0 host -> device, u(T) device -> host
    psi_host = torch.from_numpy(psi).pin_memory()
    UT_host = torch.zeros((w.ny, w.nx), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P.set_initial(psi_host)
        P.mgrit(U_T=UT_host, **kw)
    torch.cuda.synchronize(dev)
    e2e_rate, _ = whole_job_rate((time.perf_counter() - t0) / args.steps, w.space_time_updates, world, dev)
    e2e = {"value": e2e_rate, "unit": UNIT,
           "h2d_bytes_per_step": psi_host.numel() * 8, "d2h_bytes_per_step": UT_host.numel() * 8}

    # comparators on the same GPU: FP64 sequential time stepping, and FP64 MGRIT (one solve)
    seq_s = P.seq(U_T=UT)
    comparators = {"fp64_seq_timestep_gpu": w.space_time_updates / seq_s}
    fp64_iters = stats.iters
    if prec != sfde.PREC_FP64 and not args.no_fp64_comparator:
        Q = sfde.Problem(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t, w.omega,
                         precision=sfde.PREC_FP64, stream=stream.cuda_stream)
        Q.set_initial(torch.from_numpy(psi).to(dev))
        Q.set_forcing(w.forcing())
        qkw = dict(kw, rel_tol=w.rel_tol)
        Q.mgrit(U_T=UT, **qkw)
        _, qst = Q.mgrit(U_T=UT, **qkw)
        comparators["fp64_mgrit_gpu"] = w.space_time_updates / qst.seconds
        comparators["fp64_mgrit_gpu_iters"] = qst.iters
        comparators["speedup_vs_fp64_mgrit"] = value / world / comparators["fp64_mgrit_gpu"]
        fp64_iters = qst.iters
        Q.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if prec == sfde.PREC_FP64 else {"mixed-bf16": "bf16+f64", "mixed-tf32": "tf32+f64",
                                                        "mixed-auto": "bf16/tf32+f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "nt": w.nt, "beta": w.beta,
                   "gamma": w.gamma, "kx": w.kx, "ky": w.ky, "m": w.m, "rel_tol": tol,
                   "precision": args.precision, "iters": stats.iters, "levels": stats.levels,
                   "inner_vcycles": stats.inner_vcycles,
                   "coarse": ["cn", "be"][stats.coarse_used], "step_solves": stats.step_solves,
                   "l2": "space-time iterate (537 MB) larger than L2; no flush needed",
                   "parallelism": f"replicas x{world} (independent instances per GPU)"},
        "roofline": roofline,
        "kernels": kernels,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "comparators": comparators,
    }
    if rank == 0 and not args.no_cpu_baseline:
        coarse = ["cn", "be"][stats.coarse_used]
        rate, dt, cores, sample = oracle_rate(w, fp64_iters, coarse)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """The batched form: the 64 uneven instances of batch_workloads(0) (N in {63..511}, N_t in
    {256..4096}, random beta, gamma, K), mixed precision to 1e-8 with the operand type chosen per
    instance (--precision, default mixed-auto), solved by sfde_batch_solve.  value =
    sum of N_x N_y N_t over the instances / seconds per batch solve (host clock with the device
    synchronised on both sides: the instances run on 64 streams)."""
    import torch
    from sfde_workloads.generate import batch_workloads
    import paper_1805_06688_gb300 as sfde
    if not os.path.exists(sfde.library_path):
        from paper_1805_06688_gb300.build import build
        build()
    ws = batch_workloads(0, 64)
    pname = "mixed-auto" if args.precision == "mixed-bf16" else args.precision
    prec = {"mixed-bf16": sfde.PREC_MIXED_BF16, "mixed-tf32": sfde.PREC_MIXED_TF32,
            "mixed-auto": sfde.PREC_MIXED_AUTO}[pname]
    t0 = time.perf_counter()
    probs = []
    for w in ws:
        P = sfde.Problem(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, w.t(), w.omega, precision=prec)
        P.set_initial(w.initial())
        probs.append(P)
    setup_s = time.perf_counter() - t0
    kw = dict(m=8, max_levels=32, coarse=sfde.COARSE_AUTO, rel_tol=1e-8, max_iter=400)
    dofs = sum(w.space_time_updates for w in ws)
    for _ in range(args.warmup):
        sfde.batch_solve(probs, **kw)
    secs = []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, status, stats = sfde.batch_solve(probs, **kw)
            torch.cuda.synchronize()
            secs.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.median(secs)
    line = {
        "metric": METRIC, "value": dofs / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16/tf32+f64", "data": "synthetic",
        "config": {"workload": "batch64 (batch_workloads seed 0)", "instances": len(ws), "space_time_updates": dofs,
                   "m": 8, "rel_tol": 1e-8, "precision": pname, "setup_s": setup_s,
                   "converged": sum(1 for s in stats if s.converged),
                   "iters_max": max(s.iters for s in stats), "timer": "host, device synchronised",
                   "l2": "space-time iterates far larger than L2"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed-bf16", "mixed-tf32", "mixed-auto"], default="mixed-bf16")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-comparator", action="store_true")
    args = ap.parse_args()
    if args.workload == "batch64":
        return run_batch(args)
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
