"""Single-kernel probes for profiling (ncu) and timing: one building block of the solver on synthetic
data, through the library's verification hooks (include/sfde_debug.h).

  python -m paper_1805_06688_gb300.probe gemm --kind 1 --P 512 --batch 256 [--reps 5]
      one tensor-core slice GEMM Out_b = (X_b Mat)^T, batch slices of P x P times a P x P matrix
      (kind 0 BF16, 1 TF32, 2 FP32 from three TF32 products), then `reps` timed repeats;
  python -m paper_1805_06688_gb300.probe residual --n 511 --nt 256 [--digits 7] [--reps 2] [--load]
      the FP64 space-time residual of the mixed-precision solver for a random iterate (digit-split
      tensor-core products and the integer assembly), `reps` times, with a separable load if asked;
  python -m paper_1805_06688_gb300.probe p1 --n 255 --batch 64 [--reps 5]
      (M_h + tau K) U for `batch` random slices with the P1-triangle matrices of Sec. 2 (two FP64
      block-Toeplitz products per application), `reps` times.

Prints one line per probe with the device time per launch (CUDA events) where the hook reports it.
"""
from __future__ import annotations

import argparse
import ctypes as C
import sys

import numpy as np


def _gemm(args):
    import torch
    from . import _binding as B
    L = B.lib()
    L.sfde_debug_tc_gemm.argtypes = [C.c_int, C.c_void_p, C.c_longlong, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_int), C.c_int,
                                     C.POINTER(C.c_float)]
    dt = torch.bfloat16 if args.kind == 0 else torch.float32
    g = torch.Generator(device="cuda").manual_seed(1)
    P, b = args.P, args.batch
    X = torch.randn((b, P, P), device="cuda", generator=g).to(dt)
    M = torch.randn((P, P), device="cuda", generator=g).to(dt)
    O = torch.empty((b, P, P), device="cuda", dtype=dt)
    err, ms = C.c_int(0), C.c_float(0.0)
    st = L.sfde_debug_tc_gemm(args.kind, X.data_ptr(), b, 0, 1, b, P, P, M.data_ptr(), P, O.data_ptr(), C.byref(err),
                              args.reps, C.byref(ms))
    if st != 0:
        raise B.SfdeError(st, "sfde_debug_tc_gemm")
    flops = 2.0 * b * P ** 3
    nbytes = X.element_size() * (2 * b * P * P + P * P)
    print(f"gemm kind {args.kind} P {P} batch {b}: {1e3 * ms.value:.1f} us per launch, "
          f"{flops / ms.value / 1e9:.1f} TFLOP/s, {nbytes / ms.value / 1e6:.1f} GB/s")


def _residual(args):
    import time
    import torch
    from . import _binding as B
    from sfde_workloads import time_grid
    L = B.lib()
    L.sfde_debug_residual.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_double)]
    n, nt = args.n, args.nt
    Pb = B.Problem(0.55, 0.95, 1.0, 0.1, n, n, time_grid(nt), precision=B.PREC_MIXED_TF32)
    if args.load:   # the benchmark's kind of load: a Gaussian bump times sin(2 pi t), rank 1
        from sfde_workloads import gaussian_bump_forcing
        Pb.set_forcing(gaussian_bump_forcing(2, n, n, time_grid(nt))[0])
    g = torch.Generator(device="cuda").manual_seed(2)
    U = torch.randn((nt + 1, n, n), dtype=torch.float64, device="cuda", generator=g)
    rho = torch.empty((nt, n, n), dtype=torch.float32, device="cuda")
    n2 = C.c_double(0.0)
    for _ in range(args.reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = L.sfde_debug_residual(Pb.ctx, U.data_ptr(), args.digits, rho.data_ptr(), C.byref(n2))
        torch.cuda.synchronize()
        if st != 0:
            raise B.SfdeError(st, "sfde_debug_residual")
    print(f"residual n {n} nt {nt} digits {args.digits}: {1e3 * (time.perf_counter() - t0):.1f} ms per call "
          f"(host clock, scratch allocation included), ||rho||^2 = {n2.value:.6e}")


def _p1(args):
    import time
    import torch
    from . import _binding as B
    from sfde_workloads import time_grid
    L = B.lib()
    L.sfde_debug_p1_apply_S.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]
    n, b = args.n, args.batch
    Pb = B.Problem(0.8, 0.8, 3.0, 7.5, n, n, time_grid(b), operator=B.OP_P1)
    g = torch.Generator(device="cuda").manual_seed(3)
    U = torch.randn((b, n, n), dtype=torch.float64, device="cuda", generator=g)
    out = torch.empty_like(U)
    for r in range(args.reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = L.sfde_debug_p1_apply_S(Pb.ctx, U.data_ptr(), b, 1, 1, out.data_ptr())
        torch.cuda.synchronize()
        if st != 0:
            raise B.SfdeError(st, "sfde_debug_p1_apply_S")
        if r == 0:
            continue   # first call allocates the workspace
    dt = time.perf_counter() - t0
    flops = 2.0 * b * n * n * 3 * n * 2
    print(f"p1 apply n {n} batch {b}: {1e3 * dt:.3f} ms per call (host clock, pad/unpad included), "
          f"{flops / dt / 1e12:.3f} TFLOP/s of the two products")


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1805_06688_gb300.probe")
    sub = ap.add_subparsers(dest="what", required=True)
    a = sub.add_parser("gemm")
    a.add_argument("--kind", type=int, default=1, choices=[0, 1, 2])
    a.add_argument("--P", type=int, default=512)
    a.add_argument("--batch", type=int, default=256)
    a.add_argument("--reps", type=int, default=5)
    r = sub.add_parser("residual")
    r.add_argument("--n", type=int, default=511)
    r.add_argument("--nt", type=int, default=256)
    r.add_argument("--digits", type=int, default=7, choices=[4, 5, 6, 7])
    r.add_argument("--reps", type=int, default=2)
    r.add_argument("--load", action="store_true", help="with a separable load term (the FP64 combination)")
    q = sub.add_parser("p1")
    q.add_argument("--n", type=int, default=255)
    q.add_argument("--batch", type=int, default=64)
    q.add_argument("--reps", type=int, default=5)
    args = ap.parse_args(argv)
    if args.what == "gemm":
        _gemm(args)
    elif args.what == "p1":
        _p1(args)
    else:
        _residual(args)
    return 0


if __name__ == "__main__":
    sys.exit(main())
