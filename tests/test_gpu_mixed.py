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

PRECS = [("bf16", sfde.PREC_MIXED_BF16), ("tf32", sfde.PREC_MIXED_TF32)]


def _err(U, ref):
    return float(np.abs(U - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("modal", [3, 1, 0, 2])
@pytest.mark.parametrize("name,prec", PRECS)
@pytest.mark.parametrize("nx,ny,nt,m,grid,levels", [(20, 13, 64, 4, "graded", 3), (31, 31, 64, 4, "uniform", 2),
                                                     (100, 70, 96, 4, "uniform", 8)])
def test_mixed_matches_sequential(name, prec, nx, ny, nt, m, grid, levels, modal):
    """Mixed precision against the oracle's sequential solution, with the coarse levels' sweeps in the
    step's eigenbasis (modal 1, the default), every level's (modal 2), by operand type (modal 3: all
    levels with BF16, the coarse ones with TF32) and none (modal 0)."""
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
    assert L.sfde_debug_set_modal_chains(P.ctx, 4) == sfde.SFDE_EINVAL
    assert L.sfde_debug_set_modal_chains(P.ctx, -1) == sfde.SFDE_EINVAL
    assert L.sfde_debug_set_modal_chains(None, 1) == sfde.SFDE_EINVAL
    for v in (0, 2, 1, 3):
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


@pytest.mark.parametrize("name,prec", PRECS)
def test_mixed_sine_N255_Nt1024_full_size(name, prec):
    """The benchmarked workload in the bench's configuration (relative residual 1e-8), against the
    exact sequential solution at sampled time points: space-time max-norm error <= 1e-8 of max|u|
    (measured 3.7e-10)."""
    w = WORKLOADS["sine_N255_Nt1024"]
    t = w.t()
    psi = w.initial()
    P = sfde.Problem(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t, precision=prec)
    P.set_initial(psi)
    U = torch.zeros((w.nt + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    _, st = P.mgrit(U=U, m=w.m, max_levels=32, coarse=sfde.COARSE_AUTO, rel_tol=1e-8, max_iter=100)
    assert st.converged
    O = osfde.SFDE(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t)
    keep = [1, 7, 8, 100, 513, 1024]
    exact = osfde.spectral_sequential(O, psi, None, keep=keep)
    scale = np.abs(psi).max()
    for n in keep:
        assert np.abs(U[n].cpu().numpy() - exact[n]).max() < 1e-8 * scale, n


def test_mixed_bump_N511_Nt2048_full_size():
    """The N = 511 workload (padded P = 512: four-GEMM tensor-core steps and the K-grouped integer
    residual), mixed BF16 to 1e-8, against the exact sequential solution at sampled time points."""
    w = WORKLOADS["bump_N511_Nt2048"]
    t = w.t()
    psi, F = w.initial(), w.forcing()
    P = sfde.Problem(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t, precision=sfde.PREC_MIXED_BF16)
    P.set_initial(psi)
    P.set_forcing(F)
    U = torch.zeros((w.nt + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    _, st = P.mgrit(U=U, m=w.m, max_levels=32, coarse=sfde.COARSE_AUTO, rel_tol=w.rel_tol, max_iter=100)
    assert st.converged
    O = osfde.SFDE(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t)
    keep = [1, 9, 512, 1500, 2048]
    exact = osfde.spectral_sequential(O, psi, F, keep=keep)
    scale = max(np.abs(exact[n]).max() for n in keep)
    for n in keep:
        assert np.abs(U[n].cpu().numpy() - exact[n]).max() < 1e-8 * scale, n


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
