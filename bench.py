#!/usr/bin/env python
"""Throughput of the MGRIT solve of the 2-D Riesz SFDE on GB300: space-time DOF-updates/s.

One "step" is one complete MGRIT solve (all refinement steps to the stopping tolerance) of the
workload ``bump_N511_Nt2048``: N_x = N_y = 511, N_t = 2048 uniform steps on (0,1]^3,
beta = 0.55, gamma = 0.95, K_x = 1, K_y = 0.1, sixteen seeded sine modes for psi_0 and a seeded
Gaussian bump x sin(2 pi t) for f, V-cycle with m = 8, mixed precision (tensor-core V-cycles inside
FP64 refinement) stopped where the FP64 space-time residual of Eq. (2.4) falls below 1e-8 of the
initial guess's.  value = N_x N_y N_t / (device seconds per solve), summed over ranks.

Beside it, outside the timed region: the solver's execution choices picked by its autotuner, the
setup time, plain FP64 GPU MGRIT stopped by the same residual test at the same tolerance, FP64 GPU
sequential stepping, the max-norm error of the solution against the oracle's exact sequential
solution at every time point, and the oracle timed on the host cores.

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
WORKLOAD = "bump_N511_Nt2048"
REL_TOL = 1e-8
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Nominal GB300 rates (TFLOP/s): FP64 and BF16 dense; FP64 peak = measured BF16 x nominal ratio.
NOMINAL_FP64_TFLOPS = 1.25
NOMINAL_BF16_TFLOPS = 2250.0


def l2_note(w) -> str:
    """Size of the FP64 space-time iterate against the 129 MB L2 (no flush is needed above it)."""
    b = (w.nt + 1) * w.nx * w.ny * 8
    if b > 129e6:
        return f"space-time iterate ({b / 1e9:.2f} GB FP64) larger than the 129 MB L2; no flush needed"
    return f"space-time iterate ({b / 1e6:.1f} MB FP64) fits in L2: warm-cache timing"


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


# ----------------------------------------------------------------------------- oracle leg

def oracle_problem(w):
    from oracle import sfde as osfde
    prob = osfde.SFDE(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, w.t(), w.omega)
    prob.eig()
    return prob


def oracle_seq_sample(w, prob=None, steps: int | None = None, budget_s: float = 10.0):
    """The oracle's sequential FP64 time stepping (Eq. (2.4), fast-diagonalisation solve per step)
    over a bounded run of consecutive steps of the workload: its fastest path to the solution, which
    it reaches exactly (every row of Eq. (3.1) holds to rounding), so DOF-updates/s = N_x N_y x steps /
    time needs no extrapolation.  With steps None the count is sized to about budget_s seconds from
    one timed step.  Returns (rate, seconds, steps, sample text)."""
    from oracle import sfde as osfde
    prob = prob or oracle_problem(w)
    F = w.forcing()
    U = w.initial()
    t0 = time.perf_counter()
    U = prob.step(U, 1, osfde.dense_forcing(F, 1))
    one = time.perf_counter() - t0
    if steps is None:
        steps = int(min(w.nt - 1, max(8, budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    for n in range(2, 2 + steps):
        U = prob.step(U, n, osfde.dense_forcing(F, n))
    dt = time.perf_counter() - t0
    rate = w.nx * w.ny * steps / dt
    sample = (f"{steps} consecutive steps (t_2 .. t_{steps + 1}) of the oracle's FP64 sequential time stepping "
              f"(Eq. (2.4), FDM solve) on {w.name}; rate = N_x N_y x steps / time")
    return rate, dt, steps, sample


def oracle_leg(w, U_mixed, U_fp64, fp64_step_solves):
    """Oracle on the host cores (rank 0, outside the timed region): (1) the max-norm error of the GPU
    solutions against the oracle's exact sequential solution at every time point, streamed slice by
    slice; (2) the oracle's sequential stepping timed on a bounded sample; (3) one full oracle FP64
    MGRIT solve of the small manufactured workload (the anchor of the MGRIT estimate), and the oracle
    MGRIT rate on this workload estimated from the sampled step time and the step solves GPU FP64
    MGRIT took (the same algorithm)."""
    from oracle import mgrit as omgrit
    from oracle.sfde import spectral_sequential_iter
    prob = oracle_problem(w)
    acc = {}
    t0 = time.perf_counter()
    sols = [(name, U) for name, U in (("mixed", U_mixed), ("fp64_mgrit", U_fp64)) if U is not None]
    emax = {name: 0.0 for name, _ in sols}
    per_slice = dict(emax)
    smax = 0.0
    for n, E in spectral_sequential_iter(prob, w.initial(), w.forcing()):
        m = float(np.abs(E).max())
        smax = max(smax, m)
        for name, U in sols:
            d = float(np.abs(U[n] - E).max())
            emax[name] = max(emax[name], d)
            if n > 0 and m > 0:
                per_slice[name] = max(per_slice[name], d / m)
    for name, _ in sols:
        acc[name] = {"max_err_vs_oracle": emax[name] / smax, "max_err_per_slice_rel": per_slice[name],
                     "max_abs_err": emax[name], "slices_compared": w.nt + 1}
    acc["oracle_exact_s"] = time.perf_counter() - t0
    rate, dt, steps, sample = oracle_seq_sample(w, prob)
    base = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample,
            "sample_s": dt, "blas_threads": os.environ.get("OPENBLAS_NUM_THREADS", "default (all cores)")}
    step_s = dt / steps
    if fp64_step_solves:
        base["oracle_mgrit_estimate"] = {
            "value": w.space_time_updates / (step_s * fp64_step_solves), "unit": UNIT,
            "how": (f"extrapolated: sampled oracle step time x {fp64_step_solves} step solves (GPU FP64 MGRIT, same "
                    "algorithm and stopping test)")}
    a = WORKLOADS["manufactured_N31_Nt64"]
    aprob = oracle_problem(a)
    t0 = time.perf_counter()
    r = omgrit.mgrit(aprob, a.initial(), a.forcing(), m=a.m, max_levels=2, coarse="be", rel_tol=REL_TOL,
                     stop="sform")
    adt = time.perf_counter() - t0
    base["anchor"] = {"workload": a.name, "solver": "oracle FP64 MGRIT (two levels, space-time residual 1e-8)",
                      "iters": r.iters, "seconds": adt, "value": a.space_time_updates / adt, "unit": UNIT,
                      "measured": "full solve"}
    return acc, base


def run_reference(args, w):
    """The oracle timed on the host cores: each step is a bounded sample of consecutive FP64 steps of
    its sequential time stepping on the workload (see oracle_seq_sample); rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    prob = oracle_problem(w)
    _, _, steps, _ = oracle_seq_sample(w, prob, budget_s=3.0)   # sizes the sample, untimed
    rates, secs = [], []
    sample = ""
    for k in range(args.warmup + args.steps):
        rate, dt, _, sample = oracle_seq_sample(w, prob, steps=steps)
        if k >= args.warmup:
            rates.append(rate)
            secs.append(dt)
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "nt": w.nt, "m": w.m, "rel_tol": REL_TOL,
                   "solver": "FP64 CPU oracle, sequential time stepping (exact solution of Eq. (3.1))",
                   "step": f"{steps} consecutive time steps"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
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
    ("k_p1_gemm", "P1-triangle operator: block-Toeplitz FP64 products over three shifted slice copies", "alu"),
)


def roofline_from_profile(prof, lp_kind: int):
    """Roofline of the kernel class with the largest device time, plus a per-class breakdown.

    Each class's launches are timed with CUDA events inside one solve of well under a second, so the
    denominators are the measured burst rates.  FP64 SIMT GEMMs are bound by the FP64 pipe
    (measured BF16 x nominal FP64/BF16); tensor-core kernels are placed by algorithmic intensity
    against the ridge point (below it: HBM bandwidth, above it: the tensor pipe of their dtype, TF32
    at half the BF16 rate, an FP32 product of the three-product form at a sixth: three TF32 products);
    the integer assembly kernels move bytes only."""
    pk, src = peaks()
    bf16 = pk["bf16_tflops"]
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
        tc_peak = bf16 * ({1: 0.5, 2: 0.5 / 3.0}.get(lp_kind, 1.0) if k == 2 else 1.0)
        if kind == "alu":
            bound, ach, peak, unit = "alu", tfs, fp64_peak, "TFLOP/s"
            psrc = f"{src} burst BF16 {bf16} TFLOP/s x nominal FP64/BF16 {NOMINAL_FP64_TFLOPS}/{NOMINAL_BF16_TFLOPS}"
        elif kind == "hbm" or fl / by < tc_peak * 1e12 / (pk["hbm_gbs"] * 1e9):
            bound, ach, peak, unit = "hbm", gbs, pk["hbm_gbs"], "GB/s"
            psrc = f"{src} HBM copy bandwidth"
        else:
            bound, ach, peak, unit = "tensor", tfs, tc_peak, "TFLOP/s"
            psrc = f"{src} burst BF16 dense" + ({1: " x 1/2 (TF32 nominal ratio)",
                                                   2: " x 1/2 (TF32 nominal ratio) / 3 (TF32 products per FP32 product)"}
                                                  .get(lp_kind, "") if k == 2 else "")
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
    prec = {"fp64": sfde.PREC_FP64, "mixed-bf16": sfde.PREC_MIXED_BF16, "mixed-tf32": sfde.PREC_MIXED_TF32,
            "mixed-fp32": sfde.PREC_MIXED_FP32, "mixed-auto": sfde.PREC_MIXED_AUTO}[args.precision]
    t = w.t()
    psi = w.initial()
    forcing = w.forcing()
    # setup (Toeplitz coefficients, dense A, generalised eigenpairs, operands): reported, not timed
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    P = sfde.Problem(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t, w.omega, precision=prec,
                     stream=stream.cuda_stream)
    P.set_initial(torch.from_numpy(psi).to(dev))
    P.set_forcing(forcing)
    torch.cuda.synchronize(dev)
    setup_s = time.perf_counter() - t0
    # every form stops on the FP64 space-time residual of Eq. (2.4), 1e-8 of the initial guess's
    kw = dict(m=w.m, max_levels=w.max_levels, coarse=sfde.COARSE_AUTO, rel_tol=REL_TOL, max_iter=400,
              stop_kind=sfde.STOP_SFORM)
    UT = torch.zeros((w.ny, w.nx), dtype=torch.float64, device=dev)

    tuning = None
    autotune_s = 0.0
    if prec != sfde.PREC_FP64 and not args.no_autotune:
        t0 = time.perf_counter()
        tn = P.autotune(cache_path=args.tune_cache, **kw)
        autotune_s = time.perf_counter() - t0
        tuning = {"fused_pair": tn.fused_pair, "modal_chains": tn.modal_chains, "inner_cycles": tn.inner_cycles,
                  "ms": tn.ms, "seconds": autotune_s}

    def barrier():
        if world > 1:
            dist.barrier()

    stats = None
    for _ in range(args.warmup):
        _, stats = P.mgrit(U_T=UT, **kw)
    # timed region: the space-time iterate (FP64, (N_t + 1) N_x N_y x 8 B) is compared with L2 in l2_note
    P.profile_enable(False)
    barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")   # lets a profiler list the timed solves' launches alone
        ev0.record(stream)
        for _ in range(args.steps):
            _, stats = P.mgrit(U_T=UT, **kw)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
    barrier()
    launches = P.profile_read().kernel_launches
    value, sec = whole_job_rate(ev0.elapsed_time(ev1) * 1e-3 / args.steps, w.space_time_updates, world, dev)
    ms = 1e3 * sec

    # dominant kernel: per-launch CUDA-event durations over one more solve
    P.profile_enable(True)
    P.mgrit(U_T=UT, **kw)
    prof = P.profile_read()
    P.profile_enable(False)
    roofline, kernels = roofline_from_profile(prof, stats.lp_kind)

    # end to end through the C ABI with host buffers: psi_0 and the load factors host -> device,
    # u(T) device -> host, every step
    psi_host = torch.from_numpy(psi).pin_memory()
    UT_host = torch.zeros((w.ny, w.nx), dtype=torch.float64).pin_memory()
    h2d = psi_host.numel() * 8
    if forcing is not None:
        h2d += 8 * (forcing.time_w.size + forcing.bx.size + forcing.by.size)
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P.set_initial(psi_host)
        P.set_forcing(forcing)
        P.mgrit(U_T=UT_host, **kw)
    torch.cuda.synchronize(dev)
    e2e_rate, _ = whole_job_rate((time.perf_counter() - t0) / args.steps, w.space_time_updates, world, dev)
    e2e = {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": UT_host.numel() * 8}

    # the whole space-time solution of one more solve, for the error against the oracle
    want_err = rank == 0 and not args.no_cpu_baseline
    U_mixed = None
    if want_err:
        Ud = torch.empty((w.nt + 1, w.ny, w.nx), dtype=torch.float64, device=dev)
        P.mgrit(U=Ud, **kw)
        U_mixed = Ud.cpu().numpy()
        del Ud

    # comparators on the same GPU: FP64 sequential time stepping, and FP64 MGRIT stopped by the same
    # space-time residual test at the same tolerance
    seq_s = P.seq(U_T=UT)
    comparators = {"fp64_seq_timestep_gpu": w.space_time_updates / seq_s,
                   "speedup_vs_fp64_seq_timestep": value / world / (w.space_time_updates / seq_s)}
    U_fp64 = None
    fp64_step_solves = None
    if prec != sfde.PREC_FP64 and not args.no_fp64_comparator:
        Q = sfde.Problem(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t, w.omega,
                         precision=sfde.PREC_FP64, stream=stream.cuda_stream)
        Q.set_initial(torch.from_numpy(psi).to(dev))
        Q.set_forcing(forcing)
        Ud = torch.empty((w.nt + 1, w.ny, w.nx), dtype=torch.float64, device=dev) if want_err else None
        _, qst = Q.mgrit(U=Ud, U_T=UT, **kw)
        if want_err:
            U_fp64 = Ud.cpu().numpy()
            del Ud
        comparators.update({
            "fp64_mgrit_gpu": w.space_time_updates / qst.seconds, "fp64_mgrit_gpu_iters": qst.iters,
            "fp64_mgrit_stop": f"FP64 space-time residual <= {REL_TOL} x initial (same test as the mixed form)",
            "fp64_mgrit_step_solves": qst.step_solves,
            "speedup_vs_fp64_mgrit": value / world / (w.space_time_updates / qst.seconds)})
        fp64_step_solves = qst.step_solves
        Q.close()
    comparators["work_ratio_note"] = (
        "MGRIT does about 2 m/(m-1) step solves per time point per V-cycle on top of sequential stepping's one; "
        "compare the speed-ups above with that")
    dtype = "f64" if prec == sfde.PREC_FP64 else ["bf16+f64", "tf32+f64", "fp32(3xtf32)+f64"][stats.lp_kind]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "nt": w.nt, "beta": w.beta,
                   "gamma": w.gamma, "kx": w.kx, "ky": w.ky, "m": w.m, "rel_tol": REL_TOL,
                   "stop": "FP64 space-time residual of Eq. (2.4), relative to the initial guess's",
                   "precision": args.precision,
                   "operands": ["bf16", "tf32", "fp32 (3 tf32 products)"][stats.lp_kind] if stats.lp_kind >= 0 else "fp64",
                   "iters": stats.iters, "levels": stats.levels, "inner_vcycles": stats.inner_vcycles,
                   "coarse": ["cn", "be"][stats.coarse_used], "step_solves": stats.step_solves,
                   "tuning": tuning,
                   "l2": l2_note(w),
                   "parallelism": f"replicas x{world} (independent instances per GPU)"},
        "setup_s": setup_s,
        "roofline": roofline,
        "kernels": kernels,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "comparators": comparators,
    }
    if want_err:
        acc, base = oracle_leg(w, U_mixed, U_fp64, fp64_step_solves)
        line["accuracy"] = acc
        line["cpu_baseline"] = base
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
    pname = args.precision
    prec = {"mixed-bf16": sfde.PREC_MIXED_BF16, "mixed-tf32": sfde.PREC_MIXED_TF32, "mixed-fp32": sfde.PREC_MIXED_FP32,
            "mixed-auto": sfde.PREC_MIXED_AUTO}[pname]
    t0 = time.perf_counter()
    probs = []
    for w in ws:
        P = sfde.Problem(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, w.t(), w.omega, precision=prec)
        P.set_initial(w.initial())
        probs.append(P)
    setup_s = time.perf_counter() - t0
    kw = dict(m=8, max_levels=32, coarse=sfde.COARSE_AUTO, rel_tol=REL_TOL, max_iter=400, stop_kind=sfde.STOP_SFORM)
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
        "vs_baseline": None, "dtype": "+".join(sorted({["bf16", "tf32", "fp32(3xtf32)"][s.lp_kind] for s in stats
                                                       if s.lp_kind >= 0})) + "+f64",
        "data": "synthetic",
        "config": {"workload": "batch64 (batch_workloads seed 0)", "instances": len(ws), "space_time_updates": dofs,
                   "m": 8, "rel_tol": 1e-8, "precision": pname, "setup_s": setup_s,
                   "converged": sum(1 for s in stats if s.converged),
                   "iters_max": max(s.iters for s in stats), "timer": "host, device synchronised",
                   "l2": "space-time iterates far larger than L2"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


P1_WORKLOAD = "p1_example41_M32_N32768"


def run_p1(args):
    """The paper's own P1-triangle scheme (Sec. 2) on Example 4.1 in the setting of Table 2's last row:
    M = 32 intervals per direction (31^2 unknowns), tau = h^3 (N = 32768 uniform steps), K_x = 3.0,
    K_y = 7.5, beta = gamma = 0.8, solved by FP64 MGRIT on the GPU (m = 8, FCF, backward-Euler coarse
    propagator, the space-time residual of Eq. (3.1) to 1e-10 of the initial guess's), every fine
    step a CG solve preconditioned with the tensor-product spectral solve.  value = 31^2 x 32768 /
    seconds per solve (CUDA events on the library's stream); accuracy: the L2 error at T = 1 against
    the exact solution, the printed Table 2 value and the oracle's dense sequential solution."""
    import torch
    import paper_1805_06688_gb300 as sfde
    from oracle import p1 as op1
    from sfde_workloads import manufactured_exact, manufactured_initial, p1_manufactured_forcing, time_grid
    if not os.path.exists(sfde.library_path):
        from paper_1805_06688_gb300.build import build
        build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    M, beta, gamma, kx, ky = 32, 0.8, 0.8, 3.0, 7.5
    n, nt = M - 1, M ** 3
    t = time_grid(nt)
    F = p1_manufactured_forcing(n, n, t, beta, gamma, kx, ky)
    Fall = F.all()
    psi = manufactured_initial(n, n, "10exp(-t)")
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    P = sfde.Problem(beta, gamma, kx, ky, n, n, t, precision=sfde.PREC_FP64, stream=stream.cuda_stream,
                     operator=sfde.OP_P1)
    P.set_initial(torch.from_numpy(psi).to(dev))
    P.set_forcing_dense(torch.from_numpy(Fall).to(dev))
    torch.cuda.synchronize(dev)
    setup_s = time.perf_counter() - t0
    kw = dict(m=8, coarse=sfde.COARSE_BE, rel_tol=1e-10, max_iter=60, stop_kind=sfde.STOP_SFORM)
    UT = torch.zeros((n, n), dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        P.mgrit(U_T=UT, **kw)
    P.profile_enable(False)
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.nvtx.range_push("timed")
        ev0.record(stream)
        for _ in range(args.steps):
            _, stats = P.mgrit(U_T=UT, **kw)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
    launches = P.profile_read().kernel_launches
    sec = ev0.elapsed_time(ev1) * 1e-3 / args.steps
    units = n * n * nt
    value = units / sec
    P.profile_enable(True)
    P.mgrit(U_T=UT, **kw)
    prof = P.profile_read()
    P.profile_enable(False)
    roofline, kernels = roofline_from_profile(prof, -1)
    ut_gpu = UT.cpu().numpy()

    # end to end through the C ABI with host buffers: psi_0 and every load vector in, u(T) out
    psi_h = torch.from_numpy(psi).pin_memory()
    F_h = torch.from_numpy(Fall).pin_memory()
    UT_h = torch.zeros((n, n), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P.set_initial(psi_h)
        P.set_forcing_dense(F_h)
        P.mgrit(U_T=UT_h, **kw)
    torch.cuda.synchronize(dev)
    e2e = {"value": units / ((time.perf_counter() - t0) / args.steps), "unit": UNIT,
           "h2d_bytes_per_step": 8 * (psi.size + Fall.size), "d2h_bytes_per_step": 8 * n * n}

    # comparator: GPU sequential stepping with the same P1 steps, timed on the first 2048 steps (the
    # steps are uniform, so every step costs the same)
    Q = sfde.Problem(beta, gamma, kx, ky, n, n, t[:2049], precision=sfde.PREC_FP64, stream=stream.cuda_stream,
                     operator=sfde.OP_P1)
    Q.set_initial(torch.from_numpy(psi).to(dev))
    Q.set_forcing_dense(torch.from_numpy(np.ascontiguousarray(Fall[:2048])).to(dev))
    Q.seq(U_T=UT)
    seq_s = Q.seq(U_T=UT)
    Q.close()
    comparators = {"fp64_seq_timestep_gpu": n * n * 2048 / seq_s,
                   "fp64_seq_timestep_gpu_sample": "first 2048 of the 32768 uniform steps",
                   "speedup_vs_fp64_seq_timestep": value / (n * n * 2048 / seq_s),
                   "mgrit_iters": stats.iters, "levels": stats.levels, "step_solves": stats.step_solves}

    exact = lambda X, Y: manufactured_exact(X, Y, 1.0, "10exp(-t)")
    acc = {"l2_error_gpu_T1": op1.l2_error_p1(ut_gpu, exact), "table2_printed": 1.3240e-5}
    acc["ratio_to_printed"] = acc["l2_error_gpu_T1"] / acc["table2_printed"]
    base = None
    if not args.no_cpu_baseline:
        # the oracle: dense Cholesky stepping of the same P1 scheme on the host cores, all 32768 steps
        O = op1.P1SFDE(beta, gamma, kx, ky, n, n, t)
        t0 = time.perf_counter()
        ut_ref = op1.seq_timestep_p1(O, psi, F, keep_all=False)
        cpu_s = time.perf_counter() - t0
        acc["max_rel_diff_vs_oracle_T1"] = float(np.abs(ut_gpu - ut_ref).max() / np.abs(ut_ref).max())
        acc["l2_error_oracle_T1"] = op1.l2_error_p1(ut_ref, exact)
        base = {"value": units / cpu_s, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                "sample": "the whole solve: sequential stepping of the oracle's dense P1 scheme (Cholesky, "
                          f"{cpu_s:.1f} s)"}
    line = {
        "metric": "space-time DOF-updates/s to 1e-10 rel. space-time residual, P1-triangle scheme (Example 4.1, "
                  "Table 2 setting), FP64 MGRIT, 1 GB300",
        "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sec, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": P1_WORKLOAD, "operator": "P1 triangles (Sec. 2)", "nx": n, "ny": n, "nt": nt,
                   "beta": beta, "gamma": gamma, "kx": kx, "ky": ky, "m": 8, "coarse": "be", "rel_tol": 1e-10,
                   "stop": "FP64 space-time residual of Eq. (3.1), relative to the initial guess's",
                   "cg": "per step: CG to 1e-13 relative residual, preconditioned by the tensor-product spectral solve",
                   "l2": "space-time iterate 32769 x 32^2 x 8 B = 268 MB, larger than L2"},
        "setup_s": setup_s, "roofline": roofline, "kernels": kernels, "e2e": e2e, "clocks": clk.summary(),
        "gpu_launches": launches, "comparators": comparators, "accuracy": acc, "cpu_baseline": base,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed-bf16", "mixed-tf32", "mixed-fp32", "mixed-auto"],
                    default="mixed-auto")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-comparator", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tune-cache", default=None, help="autotuner cache file (a stored choice is applied untimed)")
    args = ap.parse_args()
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == P1_WORKLOAD:
        return run_p1(args)
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
