"""ctypes marshalling for ``libsfde.so`` (names and semantics follow ``include/sfde.h``)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(HERE, "libsfde.so")

(SFDE_OK, SFDE_EINVAL, SFDE_ENOMEM, SFDE_ECUDA, SFDE_ENOCONV, SFDE_ETIMEOUT, SFDE_EUNSUPPORTED,
 SFDE_ESCRATCH) = range(8)
NOALLOC_SCRATCH_DOUBLES = 5 * 262144
PREC_FP64, PREC_MIXED_BF16, PREC_MIXED_TF32, PREC_MIXED_FP32, PREC_MIXED_AUTO = 0, 1, 2, 3, 4
RELAX_FCF, RELAX_F = 0, 1
COARSE_CN, COARSE_BE, COARSE_AUTO = 0, 1, 2
OP_TENSOR, OP_P1 = 0, 1
HISTORY_MAX = 512

# every entry point declared in include/sfde.h (checked by the tests)
exported_symbols = (
    "sfde_setup", "sfde_set_initial", "sfde_set_forcing", "mgrit_solve", "seq_timestep",
    "sfde_step_batch", "sfde_step_batch_noalloc", "sfde_get_operator", "sfde_profile_enable", "sfde_profile_read",
    "sfde_destroy", "sfde_strerror", "sfde_batch_solve", "sfde_set_tuning", "sfde_get_tuning", "sfde_autotune",
    "sfde_set_forcing_dense", "sfde_two_level_bound", "sfde_choose_coarsening", "sfde_propagate_batch",
)


PROF_CLASSES = 7  # see include/sfde.h: FP64 step, FP64 residual, TC GEMM, fused step, digit products, int
# assembly, P1 operator products


class SfdeProfile(C.Structure):
    _fields_ = [("kernel_launches", C.c_longlong), ("launches", C.c_longlong * PROF_CLASSES),
                ("ms", C.c_double * PROF_CLASSES), ("flops", C.c_double * PROF_CLASSES),
                ("bytes", C.c_double * PROF_CLASSES)]


class SfdeError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {sfde_strerror(status)} (status {status})")
        self.status = status


class SfdeOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("stream", C.c_void_p), ("operator_kind", C.c_int)]


class MgritOpts(C.Structure):
    _fields_ = [("m", C.c_int), ("max_levels", C.c_int), ("min_coarse", C.c_int),
                ("relax", C.c_int), ("coarse", C.c_int), ("max_iter", C.c_int),
                ("rel_tol", C.c_double), ("abs_tol", C.c_double), ("init_seed", C.c_uint64),
                ("inner_cycles", C.c_int), ("skip_first_down", C.c_int), ("stop_kind", C.c_int)]


class SfdeTuning(C.Structure):
    _fields_ = [("fused_pair", C.c_int), ("modal_chains", C.c_int), ("inner_cycles", C.c_int),
                ("ms", C.c_double)]


class MgritStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("levels", C.c_int), ("converged", C.c_int),
                ("coarse_used", C.c_int), ("res0", C.c_double), ("res_final", C.c_double),
                ("conv_factor_last5", C.c_double), ("seconds", C.c_double), ("tub", C.c_double),
                ("step_solves", C.c_longlong), ("inner_vcycles", C.c_longlong),
                ("history", C.c_double * HISTORY_MAX), ("lp_kind", C.c_int), ("m_used", C.c_int)]

    def residual_history(self):
        return [self.history[i] for i in range(min(self.iters, HISTORY_MAX))]


_LIB = None


def lib() -> C.CDLL:
    """Load the compiled library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(library_path):
            raise RuntimeError(f"{library_path} is missing: build it with "
                               "`python -m paper_1805_06688_gb300.build` (needs nvcc)")
        L = C.CDLL(library_path)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
        L.sfde_setup.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, dp, ip, ip, dp, ip,
                                 C.POINTER(SfdeOpts), C.POINTER(vp)]
        L.sfde_set_initial.argtypes = [vp, vp]
        L.sfde_set_forcing.argtypes = [vp, ip, vp, vp, vp]
        L.sfde_set_forcing_dense.argtypes = [vp, vp]
        L.sfde_two_level_bound.argtypes = [vp, ip, ip, dp]
        L.sfde_choose_coarsening.argtypes = [vp, ip, C.c_double, C.POINTER(ip)]
        L.mgrit_solve.argtypes = [vp, C.POINTER(MgritOpts), vp, vp, C.POINTER(MgritStats)]
        L.seq_timestep.argtypes = [vp, vp, vp, dp]
        L.sfde_step_batch.argtypes = [vp, ip, ip, ip, vp, vp]
        L.sfde_step_batch_noalloc.argtypes = [vp, ip, ip, ip, vp, vp]
        L.sfde_propagate_batch.argtypes = [vp, ip, dp, ip, vp, vp, vp]
        L.sfde_get_operator.argtypes = [vp, ip, vp, vp, vp]
        L.sfde_profile_enable.argtypes = [vp, ip]
        L.sfde_profile_read.argtypes = [vp, C.POINTER(SfdeProfile)]
        L.sfde_batch_solve.argtypes = [ip, C.POINTER(vp), C.POINTER(MgritOpts), C.POINTER(vp),
                                       C.POINTER(MgritStats), C.POINTER(ip)]
        L.sfde_set_tuning.argtypes = [vp, C.POINTER(SfdeTuning)]
        L.sfde_autotune.argtypes = [vp, C.POINTER(MgritOpts), C.c_char_p, C.POINTER(SfdeTuning)]
        L.sfde_get_tuning.argtypes = [vp, C.POINTER(SfdeTuning)]
        L.sfde_destroy.argtypes = [vp]
        L.sfde_destroy.restype = None
        L.sfde_strerror.argtypes = [ip]
        L.sfde_strerror.restype = C.c_char_p
        for name in exported_symbols:
            if name not in ("sfde_destroy", "sfde_strerror"):
                getattr(L, name).restype = ip
        _LIB = L
    return _LIB


def _ptr(a):
    """Raw pointer of a NumPy array or torch tensor (None -> NULL); must be C-contiguous float64."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous float64")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("tensors must be contiguous float64")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


# (nx, ny, nt) of every live context, keyed by its address: the C side cannot check buffer sizes
_CTX_DIMS: dict[int, tuple[int, int, int]] = {}


def _ctx_key(ctx) -> int:
    return int(ctx.value if isinstance(ctx, C.c_void_p) else ctx or 0)


def _extent(a):
    """(address, bytes, is_device, device index) of a NumPy array or torch tensor."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data, a.nbytes, False, None
    if hasattr(a, "data_ptr"):
        nbytes = a.numel() * a.element_size()
        return a.data_ptr(), nbytes, bool(a.is_cuda), (a.device.index if a.is_cuda else None)
    raise TypeError(f"unsupported array type {type(a)}")


def _check_step_buffers(ctx, batch: int, src, dst, device_only: bool, where: str):
    """Refuse, before any call into C, step buffers that the kernels would read or write past their
    end (fewer than batch x N_y x N_x doubles), that overlap, or (device_only) that are not CUDA
    tensors on the current device."""
    dims = _CTX_DIMS.get(_ctx_key(ctx))
    if dims is None:
        raise ValueError(f"{where}: unknown or destroyed context")
    if src is None or dst is None:
        raise ValueError(f"{where}: src and dst are required")
    nx, ny, _ = dims
    need = int(batch) * nx * ny * 8
    if int(batch) < 1:
        raise ValueError(f"{where}: batch must be >= 1")
    exts = []
    for name, a in (("src", src), ("dst", dst)):
        _ptr(a)  # dtype and contiguity
        addr, nbytes, is_dev, dev = _extent(a)
        if nbytes < need:
            raise ValueError(f"{where}: {name} holds {nbytes // 8} doubles, needs batch x N_y x N_x = {need // 8}")
        if device_only:
            import torch
            if not is_dev:
                raise ValueError(f"{where}: {name} must be a CUDA tensor")
            if dev != torch.cuda.current_device():
                raise ValueError(f"{where}: {name} is on cuda:{dev}, the current device is "
                                 f"cuda:{torch.cuda.current_device()}")
        exts.append((addr, addr + need, is_dev))
    (a0, a1, da), (b0, b1, db) = exts
    if da == db and a0 < b1 and b0 < a1:
        raise ValueError(f"{where}: src and dst overlap")


def _check(status: int, where: str, allow=(SFDE_OK,)):
    if status not in allow:
        raise SfdeError(status, where)
    return status


def sfde_strerror(status: int) -> str:
    return lib().sfde_strerror(int(status)).decode()


def sfde_setup(beta, gamma, kx, ky, omega, nx, ny, t, precision=PREC_FP64, stream=None, operator=OP_TENSOR):
    t = np.ascontiguousarray(t, dtype=np.float64)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    opts = SfdeOpts(int(precision), stream, int(operator))
    ctx = C.c_void_p()
    st = lib().sfde_setup(float(beta), float(gamma), float(kx), float(ky),
                          om.ctypes.data_as(C.POINTER(C.c_double)), int(nx), int(ny),
                          t.ctypes.data_as(C.POINTER(C.c_double)), len(t) - 1, C.byref(opts),
                          C.byref(ctx))
    _check(st, "sfde_setup")
    _CTX_DIMS[_ctx_key(ctx)] = (int(nx), int(ny), len(t) - 1)
    return ctx


def sfde_set_initial(ctx, psi0):
    return _check(lib().sfde_set_initial(ctx, _ptr(psi0)), "sfde_set_initial")


def sfde_set_forcing(ctx, rank, time_w=None, bx=None, by=None):
    return _check(lib().sfde_set_forcing(ctx, int(rank), _ptr(time_w), _ptr(bx), _ptr(by)),
                  "sfde_set_forcing")


def sfde_set_forcing_dense(ctx, F=None):
    """F: (N_t, N_y, N_x) float64 (host or device), or None to clear the load."""
    if F is not None:
        dims = _CTX_DIMS.get(_ctx_key(ctx))
        if dims is None:
            raise ValueError("sfde_set_forcing_dense: unknown or destroyed context")
        nx, ny, nt = dims
        _ptr(F)
        if tuple(F.shape) != (nt, ny, nx):
            raise ValueError(f"sfde_set_forcing_dense: F has shape {tuple(F.shape)}, needs {(nt, ny, nx)}")
    return _check(lib().sfde_set_forcing_dense(ctx, _ptr(F)), "sfde_set_forcing_dense")


def mgrit_solve(ctx, opts: MgritOpts | None, U=None, U_T=None, check=True):
    stats = MgritStats()
    st = lib().mgrit_solve(ctx, C.byref(opts) if opts is not None else None, _ptr(U), _ptr(U_T),
                           C.byref(stats))
    if check:
        _check(st, "mgrit_solve")
    return st, stats


def seq_timestep(ctx, U=None, U_T=None):
    sec = C.c_double(0.0)
    _check(lib().seq_timestep(ctx, _ptr(U), _ptr(U_T), C.byref(sec)), "seq_timestep")
    return sec.value


def sfde_batch_solve(ctxs, opts: MgritOpts | None, U_T=None, check=True):
    """Solve independent instances concurrently; returns (status, per-instance statuses, stats)."""
    n = len(ctxs)
    carr = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    uarr = None
    if U_T is not None:
        uarr = (C.c_void_p * n)(*[_ptr(u) for u in U_T])
    stats = (MgritStats * n)()
    status = (C.c_int * n)()
    st = lib().sfde_batch_solve(n, carr, C.byref(opts) if opts is not None else None, uarr, stats, status)
    if check:
        _check(st, "sfde_batch_solve", allow=(SFDE_OK, SFDE_ENOCONV))
    return st, list(status), list(stats)


def sfde_step_batch(ctx, n0, dn, batch, src, dst):
    """src, dst: at least batch x N_y x N_x doubles each, host or device, not overlapping
    (ValueError otherwise, before any call into the library)."""
    _check_step_buffers(ctx, batch, src, dst, False, "sfde_step_batch")
    return _check(lib().sfde_step_batch(ctx, int(n0), int(dn), int(batch), _ptr(src), _ptr(dst)),
                  "sfde_step_batch")


def sfde_propagate_batch(ctx, scheme, dts, src, dst, g=None):
    """dst[b] = Psi(dts[b]) src[b] + g[b] (coarse propagator CN or BE, no load); src, g, dst: at least
    len(dts) x N_y x N_x doubles each (ValueError otherwise, before any call into the library)."""
    dts = np.ascontiguousarray(dts, dtype=np.float64)
    batch = len(dts)
    _check_step_buffers(ctx, batch, src, dst, False, "sfde_propagate_batch")
    if g is not None:
        _check_step_buffers(ctx, batch, g, dst, False, "sfde_propagate_batch")
    return _check(lib().sfde_propagate_batch(ctx, int(scheme), dts.ctypes.data_as(C.POINTER(C.c_double)), batch,
                                             _ptr(src), _ptr(g), _ptr(dst)), "sfde_propagate_batch")


def sfde_step_batch_noalloc(ctx, n0, dn, batch, src, dst):
    """Queue the batched step on the context's stream using the library's fixed device scratch
    (no device allocation).  src and dst: CUDA tensors on the current device holding at least
    batch x N_y x N_x doubles each, not overlapping (ValueError otherwise, before any call into the
    library).  Returns the raw status."""
    _check_step_buffers(ctx, batch, src, dst, True, "sfde_step_batch_noalloc")
    return lib().sfde_step_batch_noalloc(ctx, int(n0), int(dn), int(batch), _ptr(src), _ptr(dst))


def sfde_get_operator(ctx, direction, n):
    coeffs = np.zeros(n)
    lam = np.zeros(n)
    V = np.zeros((n, n))
    _check(lib().sfde_get_operator(ctx, int(direction), _ptr(coeffs), _ptr(lam), _ptr(V)),
           "sfde_get_operator")
    return coeffs, lam, V


def sfde_profile_enable(ctx, enable: bool):
    return _check(lib().sfde_profile_enable(ctx, int(bool(enable))), "sfde_profile_enable")


def sfde_profile_read(ctx) -> SfdeProfile:
    p = SfdeProfile()
    _check(lib().sfde_profile_read(ctx, C.byref(p)), "sfde_profile_read")
    return p


def sfde_set_tuning(ctx, fused_pair=1, modal_chains=1, inner_cycles=0):
    t = SfdeTuning(int(fused_pair), int(modal_chains), int(inner_cycles), 0.0)
    _check(lib().sfde_set_tuning(ctx, C.byref(t)), "sfde_set_tuning")


def sfde_get_tuning(ctx) -> SfdeTuning:
    t = SfdeTuning()
    _check(lib().sfde_get_tuning(ctx, C.byref(t)), "sfde_get_tuning")
    return t


def sfde_autotune(ctx, opts: MgritOpts, cache_path=None) -> SfdeTuning:
    t = SfdeTuning()
    path = None if cache_path is None else os.fsencode(cache_path)
    _check(lib().sfde_autotune(ctx, C.byref(opts), path, C.byref(t)), "sfde_autotune")
    return t


def sfde_destroy(ctx):
    if ctx:
        _CTX_DIMS.pop(_ctx_key(ctx), None)
        lib().sfde_destroy(ctx)


def batch_solve(problems, U_T=None, check=True, **kw):
    """sfde_batch_solve over a list of Problem objects (shared options as for Problem.mgrit)."""
    return sfde_batch_solve([p.ctx for p in problems], make_opts(**kw), U_T, check=check)


STOP_NATIVE, STOP_SFORM = 0, 1


def make_opts(m=2, max_levels=64, min_coarse=2, relax=RELAX_FCF, coarse=COARSE_AUTO, max_iter=100,
              rel_tol=1e-10, abs_tol=0.0, init_seed=0, inner_cycles=0, skip_first_down=False,
              stop_kind=STOP_NATIVE) -> MgritOpts:
    return MgritOpts(int(m), int(max_levels), int(min_coarse), int(relax), int(coarse),
                     int(max_iter), float(rel_tol), float(abs_tol), int(init_seed), int(inner_cycles),
                     int(bool(skip_first_down)), int(stop_kind))


class Problem:
    """Owning wrapper around one ``sfde_ctx`` (destroyed with the object)."""

    def __init__(self, beta, gamma, kx, ky, nx, ny, t, omega=(0.0, 1.0, 0.0, 1.0),
                 precision=PREC_FP64, stream=None, operator=OP_TENSOR):
        self.nx, self.ny = int(nx), int(ny)
        self.t = np.ascontiguousarray(t, dtype=np.float64)
        self.nt = len(self.t) - 1
        self.ctx = sfde_setup(beta, gamma, kx, ky, omega, nx, ny, self.t, precision, stream, operator)

    def set_initial(self, psi0):
        sfde_set_initial(self.ctx, psi0)

    def set_forcing(self, forcing):
        """``forcing``: an object with time_w (N_t, R), bx (R, N_x), by (R, N_y), or None."""
        if forcing is None:
            sfde_set_forcing(self.ctx, 0)
            return
        tw = np.ascontiguousarray(forcing.time_w, dtype=np.float64)
        bx = np.ascontiguousarray(forcing.bx, dtype=np.float64)
        by = np.ascontiguousarray(forcing.by, dtype=np.float64)
        sfde_set_forcing(self.ctx, tw.shape[1], tw, bx, by)

    def two_level_bound(self, m, coarse=COARSE_CN):
        """Theorem 3.1's bound (Eq. (3.11)) for coarsening factor m, evaluated on the device."""
        b = C.c_double()
        _check(lib().sfde_two_level_bound(self.ctx, int(m), int(coarse), C.byref(b)), "sfde_two_level_bound")
        return b.value

    def choose_coarsening(self, coarse=COARSE_AUTO, rel_tol=1e-10):
        """The coarsening factor mgrit uses with m = 0."""
        m = C.c_int()
        _check(lib().sfde_choose_coarsening(self.ctx, int(coarse), float(rel_tol), C.byref(m)),
               "sfde_choose_coarsening")
        return m.value

    def set_forcing_dense(self, F):
        """F: (N_t, N_y, N_x) array of load vectors (host or device), or None."""
        sfde_set_forcing_dense(self.ctx, F)

    def mgrit(self, U=None, U_T=None, check=True, **kw):
        return mgrit_solve(self.ctx, make_opts(**kw), U, U_T, check=check)

    def seq(self, U=None, U_T=None):
        return seq_timestep(self.ctx, U, U_T)

    def step_batch(self, n0, dn, src, dst):
        return sfde_step_batch(self.ctx, n0, dn, src.shape[0], src, dst)

    def operator(self, direction):
        return sfde_get_operator(self.ctx, direction, self.nx if direction == 0 else self.ny)

    def set_tuning(self, fused_pair=1, modal_chains=1, inner_cycles=0):
        sfde_set_tuning(self.ctx, fused_pair, modal_chains, inner_cycles)

    def tuning(self) -> SfdeTuning:
        return sfde_get_tuning(self.ctx)

    def autotune(self, cache_path=None, **kw) -> SfdeTuning:
        """Times the solver's execution choices on this problem with the options ``kw`` (as for
        ``mgrit``) and keeps the fastest; overwrites the iterate."""
        return sfde_autotune(self.ctx, make_opts(**kw), cache_path)

    def profile_enable(self, enable=True):
        sfde_profile_enable(self.ctx, enable)

    def profile_read(self) -> SfdeProfile:
        return sfde_profile_read(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            sfde_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
