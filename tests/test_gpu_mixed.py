"""Mixed-precision MGRIT (BF16 / TF32 tensor-core V-cycles inside FP64 iterative refinement)
against the FP64 oracle.  Acceptance: max-norm error <= 1e-8 relative to the max norm of the
space-time solution, at every time point, against the exact sequential solution of Eq. (2.4)."""
import ctypes

import numpy as np
import pytest

from oracle import sfde as osfde
from sfde_workloads import WORKLOADS, gaussian_bump_forcing, sine_mode_amplitudes, sine_mode_nodal, time_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_06688_gb300 as sfde  # noqa: E402

PRECS = [("bf16", sfde.PREC_MIXED_BF16), ("tf32", sfde.PREC_MIXED_TF32), ("fp32", sfde.PREC_MIXED_FP32)]


def _err(U, ref):
    return float(np.abs(U - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("modal", [3, 1, 0, 2, 4])
@pytest.mark.parametrize("name,prec", PRECS)
@pytest.mark.parametrize("nx,ny,nt,m,grid,levels", [(20, 13, 64, 4, "graded", 3), (31, 31, 64, 4, "uniform", 2),
                                                     (100, 70, 96, 4, "uniform", 8)])
def test_mixed_matches_sequential(name, prec, nx, ny, nt, m, grid, levels, modal):
    """Mixed precision against the oracle's sequential solution, with the coarse levels' sweeps in the
    step's eigenbasis (modal 1, the default), every level's (modal 2), by operand type (modal 3: all
    levels with BF16, the coarse ones with TF32), none (modal 0), and the whole inner solve in the
    eigenbasis (modal 4; with BF16 storage as modal 1)."""
    t = time_grid(nt, 1.0, grid)
    F, _ = gaussian_bump_forcing(5, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(4), nx, ny)
    P = sfde.Problem(0.6, 0.9, 1.0, 0.5, nx, ny, t, precision=prec)
    L = sfde.lib()
    L.sfde_debug_set_modal_chains.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert L.sfde_debug_set_modal_chains(P.ctx, modal) == 0
    P.set_initial(psi)
    P.set_forcing(F)
    U = np.zeros((nt + 1, ny, nx))
    _, st = P.mgrit(U=U, m=m, max_levels=levels, coarse=sfde.COARSE_BE, rel_tol=1e-11, max_iter=60)
    O = osfde.SFDE(0.6, 0.9, 1.0, 0.5, nx, ny, t)
    ref = osfde.seq_timestep(O, psi, F)
    assert st.converged
    assert _err(U, ref) < 1e-8, (st.iters, st.inner_vcycles, _err(U, ref))


def test_modal_chains_setting_range():
    P = sfde.Problem(0.6, 0.9, 1.0, 0.5, 31, 31, time_grid(16, 1.0, "uniform"), precision=sfde.PREC_MIXED_BF16)
    L = sfde.lib()
    L.sfde_debug_set_modal_chains.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert L.sfde_debug_set_modal_chains(P.ctx, 5) == sfde.SFDE_EINVAL
    assert L.sfde_debug_set_modal_chains(P.ctx, -1) == sfde.SFDE_EINVAL
    assert L.sfde_debug_set_modal_chains(None, 1) == sfde.SFDE_EINVAL
    for v in (0, 2, 1, 3, 4):
        assert L.sfde_debug_set_modal_chains(P.ctx, v) == 0


@pytest.mark.parametrize("name,prec", PRECS)
def test_mixed_manufactured(name, prec):
    w = WORKLOADS["manufactured_N31_Nt64"]
    t = w.t()
    P = sfde.Problem(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t, precision=prec)
    P.set_initial(w.initial())
    P.set_forcing(w.forcing())
    U = np.zeros((w.nt + 1, w.ny, w.nx))
    _, st = P.mgrit(U=U, m=w.m, max_levels=2, coarse=sfde.COARSE_BE, rel_tol=1e-11, max_iter=60)
    ref = osfde.seq_timestep(osfde.SFDE(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t), w.initial(), w.forcing())
    assert st.converged and _err(U, ref) < 1e-8


def _all_slice_errors(U, O, psi, F):
    """Max-norm error of every time slice of U (a device tensor) against the oracle's exact
    sequential solution, streamed slice by slice: (max |U - u| / max |u| over space-time,
    max over n >= 1 of max |U_n - u_n| / max |u_n|)."""
    Uh = U.cpu().numpy()
    emax = smax = per = 0.0
    for n, E in osfde.spectral_sequential_iter(O, psi, F):
        d, m = float(np.abs(Uh[n] - E).max()), float(np.abs(E).max())
        emax, smax = max(emax, d), max(smax, m)
        if n > 0 and m > 0:
            per = max(per, d / m)
    return emax / smax, per


@pytest.mark.parametrize("name,prec", PRECS)
def test_mixed_sine_N255_Nt1024_full_size(name, prec):
    """The N = 255 workload (f = 0, u decays by about 1e-7 up to T) at full size, stopped on the FP64
    space-time residual at 1e-8, against the exact sequential solution at all 1025 time points:
    space-time max-norm error <= 1e-8 of max|u|; the error relative to each slice's own maximum is
    bounded too (the late slices are 1e-7 of the first)."""
    w = WORKLOADS["sine_N255_Nt1024"]
    t = w.t()
    psi = w.initial()
    P = sfde.Problem(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t, precision=prec)
    P.set_initial(psi)
    U = torch.zeros((w.nt + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    _, st = P.mgrit(U=U, m=w.m, max_levels=32, coarse=sfde.COARSE_AUTO, rel_tol=1e-8, max_iter=100)
    assert st.converged
    O = osfde.SFDE(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t)
    glob, per = _all_slice_errors(U, O, psi, None)
    print(f"sine_N255_Nt1024 {name}: space-time {glob:.2e}, worst slice-relative {per:.2e}")
    assert glob < 1e-8, glob
    assert per < 1e-4, per


@pytest.mark.parametrize("name,prec,modal,ic", [(n, p, 2, 3) for n, p in PRECS] +
                         [("tf32", sfde.PREC_MIXED_TF32, 4, 5), ("tf32", sfde.PREC_MIXED_TF32, 4, 8),
                          ("fp32", sfde.PREC_MIXED_FP32, 4, 3)])
def test_mixed_bump_N511_Nt2048_full_size(name, prec, modal, ic):
    """The N = 511 workload (padded P = 512: four-GEMM tensor-core steps and the K-grouped integer
    residual), stopped on the FP64 space-time residual at 1e-8 with the fine level's F-relaxations in
    the eigenbasis and 3 V-cycles per refinement step, or the whole inner solve in the eigenbasis
    (modal 4) with 3 to 8 V-cycles, against the exact sequential solution at all 2049 time points."""
    w = WORKLOADS["bump_N511_Nt2048"]
    t = w.t()
    psi, F = w.initial(), w.forcing()
    P = sfde.Problem(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t, precision=prec)
    P.set_initial(psi)
    P.set_forcing(F)
    P.set_tuning(fused_pair=1, modal_chains=modal, inner_cycles=ic)
    U = torch.zeros((w.nt + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    _, st = P.mgrit(U=U, m=w.m, max_levels=32, coarse=sfde.COARSE_AUTO, rel_tol=1e-8, max_iter=100,
                    stop_kind=sfde.STOP_SFORM)
    assert st.converged
    O = osfde.SFDE(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t)
    glob, per = _all_slice_errors(U, O, psi, F)
    print(f"bump_N511_Nt2048 {name} modal {modal} ic {ic}: {st.iters} steps, {st.seconds * 1e3:.1f} ms, "
          f"space-time {glob:.2e}, worst slice-relative {per:.2e}")
    assert glob < 1e-8, glob
    assert per < 1e-6, per


def test_mixed_adaptive_and_exact_residual_digits_agree():
    """The refinement with per-iteration residual digits (4 to 7) and with 7 throughout both reach
    the exact sequential solution to 1e-8; the stopping test always uses 7 digits."""
    import ctypes
    nx, ny, nt = 100, 70, 96
    t = time_grid(nt, 1.0, "uniform")
    F, _ = gaussian_bump_forcing(5, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(4), nx, ny)
    ref = osfde.seq_timestep(osfde.SFDE(0.6, 0.9, 1.0, 0.5, nx, ny, t), psi, F)
    L = sfde.lib()
    L.sfde_debug_set_residual_digits.argtypes = [ctypes.c_void_p, ctypes.c_int]
    for nd in (0, 7):
        P = sfde.Problem(0.6, 0.9, 1.0, 0.5, nx, ny, t, precision=sfde.PREC_MIXED_BF16)
        P.set_initial(psi)
        P.set_forcing(F)
        assert L.sfde_debug_set_residual_digits(P.ctx, nd) == 0
        U = np.zeros((nt + 1, ny, nx))
        _, st = P.mgrit(U=U, m=4, max_levels=8, coarse=sfde.COARSE_BE, rel_tol=1e-11, max_iter=60)
        assert st.converged
        assert _err(U, ref) < 1e-8, (nd, st.iters, _err(U, ref))


@pytest.mark.parametrize("name,prec", PRECS)
def test_mixed_skip_first_down_and_space_time_stop(name, prec):
    """Mixed precision with the first V-cycle of every inner solve skipping its down-cycle
    relaxation (a separately captured graph), stopping on the space-time residual: the result still
    matches the exact sequential solution to 1e-8, at every time point."""
    nx, ny, nt = 100, 70, 96
    t = time_grid(nt, 1.0, "uniform")
    F, _ = gaussian_bump_forcing(5, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(4), nx, ny)
    ref = osfde.seq_timestep(osfde.SFDE(0.6, 0.9, 1.0, 0.5, nx, ny, t), psi, F)
    P = sfde.Problem(0.6, 0.9, 1.0, 0.5, nx, ny, t, precision=prec)
    P.set_initial(psi)
    P.set_forcing(F)
    for skip in (True, False):
        U = np.zeros((nt + 1, ny, nx))
        _, st = P.mgrit(U=U, m=4, max_levels=8, coarse=sfde.COARSE_BE, rel_tol=1e-11, max_iter=60,
                        skip_first_down=skip, stop_kind=sfde.STOP_SFORM)
        assert st.converged
        assert _err(U, ref) < 1e-8, (skip, st.iters, _err(U, ref))


@pytest.mark.parametrize("name,prec", PRECS)
def test_mixed_dense_forcing(name, prec):
    """Mixed precision with a dense (non-separable) load: the FP64 residual adds F_n slice by slice;
    the result matches the exact sequential solution to 1e-8 at every time point."""
    from sfde_workloads import moving_bump_dense_forcing
    nx, ny, nt = 100, 70, 96
    t = time_grid(nt, 1.0, "graded")
    D, _ = moving_bump_dense_forcing(11, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(4), nx, ny)
    ref = osfde.seq_timestep(osfde.SFDE(0.6, 0.9, 1.0, 0.5, nx, ny, t), psi, D)
    P = sfde.Problem(0.6, 0.9, 1.0, 0.5, nx, ny, t, precision=prec)
    P.set_initial(psi)
    P.set_forcing_dense(D.F)
    U = np.zeros((nt + 1, ny, nx))
    _, st = P.mgrit(U=U, m=4, max_levels=8, coarse=sfde.COARSE_BE, rel_tol=1e-11, max_iter=60)
    assert st.converged
    assert _err(U, ref) < 1e-8, (st.iters, _err(U, ref))


@pytest.mark.parametrize("name,prec", PRECS)
def test_mixed_shishkin_grid(name, prec):
    """Mixed precision on the piecewise-uniform partition of Sec. 4.1 (three different step sizes,
    so the fine propagator changes along the grid): exact sequential solution to 1e-8 at every
    time point."""
    nx, ny, nt = 100, 70, 128
    t = time_grid(nt, 1.0, "shishkin", eps=2.0 ** -6)
    F, _ = gaussian_bump_forcing(5, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(4), nx, ny)
    ref = osfde.seq_timestep(osfde.SFDE(0.6, 0.7, 3.0, 7.5, nx, ny, t), psi, F)
    P = sfde.Problem(0.6, 0.7, 3.0, 7.5, nx, ny, t, precision=prec)
    P.set_initial(psi)
    P.set_forcing(F)
    U = np.zeros((nt + 1, ny, nx))
    _, st = P.mgrit(U=U, m=4, max_levels=8, coarse=sfde.COARSE_AUTO, rel_tol=1e-11, max_iter=60)
    assert st.converged
    assert _err(U, ref) < 1e-8, (st.iters, _err(U, ref))


def test_mixed_graded_N1023_Nt4096_full_size():
    """The largest workload: 1023^2 nodes (padded P = 1024, dense 1023 x 1023 Toeplitz matrices),
    4096 steps on the graded grid t_n = (n/N)^2 (the fine propagator changes at every step), m = 16,
    operands chosen by SFDE_PREC_MIXED_AUTO (FP32 here, inner solve in the eigenbasis), stopped on the
    FP64 space-time residual at 1e-8.  Against the exact sequential solution at every C-point of the
    fine level (every 16th time point) and at the first 16 steps, where the grid's steps are
    smallest."""
    w = WORKLOADS["graded_N1023_Nt4096"]
    t = w.t()
    psi, F = w.initial(), w.forcing()
    P = sfde.Problem(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t, precision=sfde.PREC_MIXED_AUTO)
    P.set_initial(psi)
    P.set_forcing(F)
    U = torch.zeros((w.nt + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    _, st = P.mgrit(U=U, m=w.m, max_levels=32, coarse=sfde.COARSE_AUTO, rel_tol=1e-8, max_iter=100,
                    stop_kind=sfde.STOP_SFORM)
    assert st.converged and st.lp_kind == 2
    keep = sorted(set(range(0, w.nt + 1, w.m)) | set(range(1, 17)))
    Uk = U[torch.tensor(keep, device="cuda")].cpu().numpy()
    del U
    pos = {n: k for k, n in enumerate(keep)}
    O = osfde.SFDE(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t)
    emax = smax = 0.0
    for n, E in osfde.spectral_sequential_iter(O, psi, F, keep=keep):
        emax = max(emax, float(np.abs(Uk[pos[n]] - E).max()))
        smax = max(smax, float(np.abs(E).max()))
    print(f"graded_N1023_Nt4096: {st.iters} refinement steps, error {emax / smax:.2e} of max|u|")
    assert emax <= 1e-8 * smax, emax / smax
