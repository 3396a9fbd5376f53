"""The FP64 space-time residual of the mixed-precision solver against the oracle's definition
rho_n = F_n + B_n U_{n-1} - S_n U_n (Eq. (2.4)), for both ways of forming it: FP64 arithmetic,
and exact integer arithmetic around digit-split BF16 tensor-core products (fixed point on a grid
of 2^-54 of each pair of time slices' maximum; contractions longer than 256 in groups of 256).

The residual is formed to FP64-product accuracy: where U nearly solves the system its norm is a
small difference of terms of size ||S U||, and must still agree with the oracle to 1e-11 ||S U||.
The norm itself only decides when Algorithm 1 stops, so the tensor-core path sums the squares of
the stored FP32 values (FP32 over four values, FP64 beyond): 2^-20 of ||rho|| is allowed on top.
The stored values are TF32 (10-bit mantissa), checked to 2^-10.
"""
import ctypes

import numpy as np
import pytest

from oracle import sfde as osfde
from sfde_workloads import gaussian_bump_forcing, sine_mode_amplitudes, sine_mode_nodal, time_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_06688_gb300 as sfde  # noqa: E402


def call_residual(P, U, use_tc):
    L = sfde.lib()
    L.sfde_debug_residual.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_double)]
    nt = U.shape[0] - 1
    rho = np.zeros((nt,) + U.shape[1:], dtype=np.float32)
    n2 = ctypes.c_double(0)
    st = L.sfde_debug_residual(P.ctx, U.ctypes.data, int(use_tc), rho.ctypes.data, ctypes.byref(n2))
    return st, rho, np.sqrt(n2.value)


def gpu_residual(P, U, use_tc):
    st, rho, nrm = call_residual(P, U, use_tc)
    assert st == 0, sfde.sfde_strerror(st)
    return rho, nrm


def oracle_residual(O, U, F):
    rho, su = [], []
    for n in range(1, O.nt + 1):
        tau = 0.5 * (O.t[n] - O.t[n - 1])
        r = O.apply_B(U[n - 1], tau) - O.apply_S(U[n], tau)
        if F is not None:
            r = r + F.dense(n)
        rho.append(r)
        su.append(np.sum(O.apply_S(U[n], tau) ** 2))
    return np.stack(rho), np.sqrt(sum(su))


@pytest.mark.parametrize("use_tc", [0, 1])
@pytest.mark.parametrize("nx,ny,nt,near", [(50, 70, 16, False), (255, 200, 6, False), (31, 31, 12, True),
                                           (450, 500, 3, True), (1000, 700, 2, False)])
def test_residual_matches_oracle(use_tc, nx, ny, nt, near):
    t = time_grid(nt, 1.0, "graded")
    F, _ = gaussian_bump_forcing(8, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(6), nx, ny)
    O = osfde.SFDE(0.65, 0.85, 1.2, 0.6, nx, ny, t)
    rng = np.random.default_rng(nx + nt)
    if near:   # an iterate that almost solves the system: the residual is a small difference
        U = osfde.seq_timestep(O, psi, F) + 1e-9 * rng.standard_normal((nt + 1, ny, nx))
        U[0] = psi
    else:
        U = rng.standard_normal((nt + 1, ny, nx))
    P = sfde.Problem(0.65, 0.85, 1.2, 0.6, nx, ny, t, precision=sfde.PREC_MIXED_TF32)
    P.set_forcing(F)
    if use_tc and min(nx, ny) <= 32:
        # one 32-wide tile per direction: below the digit products' 64-column tile (the solver takes
        # the FP64 residual there)
        st, _, _ = call_residual(P, np.ascontiguousarray(U), use_tc)
        assert st == sfde.SFDE_EUNSUPPORTED, sfde.sfde_strerror(st)
        return
    rho, nrm = gpu_residual(P, np.ascontiguousarray(U), use_tc)
    ref, scale = oracle_residual(O, U, F)
    rn = np.sqrt(np.sum(ref ** 2))
    assert abs(nrm - rn) <= 1e-11 * scale + 2.0 ** -20 * rn, (nrm, rn, scale)
    tol = 2.0 ** -10 * np.abs(ref).max(axis=(1, 2), keepdims=True) + 1e-13 * scale
    assert np.all(np.abs(rho - ref) <= tol)


@pytest.mark.parametrize("use_tc", [0, 1])
def test_residual_wide_dynamic_range(use_tc):
    """Values spread over eight decades inside each slice, slices of very different size (and one
    exactly zero): the fixed-point grid follows each pair of slices, so the residual still agrees
    with the oracle to FP64-product accuracy."""
    nx, ny, nt = 60, 45, 10
    t = time_grid(nt, 1.0, "uniform")
    O = osfde.SFDE(0.8, 0.7, 1.0, 2.0, nx, ny, t)
    rng = np.random.default_rng(7)
    U = rng.standard_normal((nt + 1, ny, nx)) * 10.0 ** rng.uniform(-8, 0, (nt + 1, ny, nx))
    U *= 10.0 ** rng.uniform(-20, 20, (nt + 1, 1, 1))
    U[4] = 0.0
    P = sfde.Problem(0.8, 0.7, 1.0, 2.0, nx, ny, t, precision=sfde.PREC_MIXED_TF32)
    rho, nrm = gpu_residual(P, np.ascontiguousarray(U), use_tc)
    ref, scale = oracle_residual(O, U, None)
    rn = np.sqrt(np.sum(ref ** 2))
    assert abs(nrm - rn) <= 1e-11 * scale + 2.0 ** -20 * rn
    # per time point: error relative to that step's own terms
    for n in range(nt):
        tau = 0.5 * (t[n + 1] - t[n])
        terms = np.sqrt(np.sum(O.apply_B(U[n], tau) ** 2) + np.sum(O.apply_S(U[n + 1], tau) ** 2))
        assert np.sqrt(np.sum((rho[n] - ref[n]) ** 2)) <= 2.0 ** -10 * np.sqrt(np.sum(ref[n] ** 2)) + 1e-12 * terms


def test_residual_not_finite():
    """A non-finite iterate gives a non-finite residual norm (the solver's divergence check)."""
    nx, ny, nt = 40, 40, 6
    t = time_grid(nt, 1.0, "uniform")
    U = np.random.default_rng(1).standard_normal((nt + 1, ny, nx))
    U[3, 5, 7] = np.inf
    P = sfde.Problem(0.8, 0.7, 1.0, 2.0, nx, ny, t, precision=sfde.PREC_MIXED_TF32)
    _, nrm = gpu_residual(P, U, 1)
    assert not np.isfinite(nrm)


@pytest.mark.parametrize("nd", [4, 5, 6])
def test_residual_with_fewer_digits(nd):
    """With nd digits per operand the products are truncated at about 2^(9 - 8 nd) of the operands'
    scale (the refinement uses this while its residual is still large); the error against the
    oracle is bounded by 2^(12 - 8 nd) of ||S U|| (a factor 8 of margin), and shrinks with nd."""
    nx, ny, nt = 255, 200, 4
    t = time_grid(nt, 1.0, "uniform")
    O = osfde.SFDE(0.65, 0.85, 1.2, 0.6, nx, ny, t)
    U = np.random.default_rng(nd).standard_normal((nt + 1, ny, nx))
    P = sfde.Problem(0.65, 0.85, 1.2, 0.6, nx, ny, t, precision=sfde.PREC_MIXED_TF32)
    rho, nrm = gpu_residual(P, U, nd)
    ref, scale = oracle_residual(O, U, None)
    rn = np.sqrt(np.sum(ref ** 2))
    assert abs(nrm - rn) <= 2.0 ** (12 - 8 * nd) * scale + 2.0 ** -20 * rn


def test_residual_of_a_zero_iterate_is_the_load():
    """Pairs of zero slices have no fixed-point unit, and a tiny slice makes the unit so fine that the
    load does not fit the 128-bit integer sum: the combination keeps the FP64 form there, so
    rho_n = F_n (n >= 2) and rho_1 = F_1 + B_1 psi_0 (the integer form with the load) still agree with
    the oracle to FP32 storage accuracy."""
    nx, ny, nt = 130, 96, 5
    t = time_grid(nt, 1.0, "uniform")
    F, _ = gaussian_bump_forcing(3, nx, ny, t)
    O = osfde.SFDE(0.7, 0.75, 1.0, 0.4, nx, ny, t)
    U = np.zeros((nt + 1, ny, nx))
    U[0] = sine_mode_nodal(sine_mode_amplitudes(2), nx, ny)
    U[3] = 1e-300 * np.random.default_rng(4).standard_normal((ny, nx))   # tiny but nonzero
    P = sfde.Problem(0.7, 0.75, 1.0, 0.4, nx, ny, t, precision=sfde.PREC_MIXED_FP32)   # plain FP32 output
    P.set_forcing(F)
    rho, nrm = gpu_residual(P, np.ascontiguousarray(U), 1)
    ref, scale = oracle_residual(O, U, F)
    for n in range(nt):
        assert np.abs(rho[n] - ref[n]).max() <= 2.0 ** -20 * np.abs(ref[n]).max(), n
    assert abs(nrm - np.sqrt(np.sum(ref ** 2))) <= 2.0 ** -20 * np.sqrt(np.sum(ref ** 2))


@pytest.mark.parametrize("prec", [sfde.PREC_MIXED_TF32, sfde.PREC_MIXED_FP32])
def test_first_residual_of_the_solver_takes_the_load_for_zero_pairs(prec):
    """The solver's first iterate is psi_0 followed by zeros: it forms the digit products for the pair
    (psi_0, U_1 = 0) alone and takes rho_n = F_n for n >= 2 without reading any product.  Its norm
    (the first entry of the residual history, 4 digits) equals the general form's on the same
    iterate to the bit, and the oracle's within the 4-digit truncation and FP32 storage."""
    nx, ny, nt = 130, 96, 40
    t = time_grid(nt, 1.0, "graded")
    F, _ = gaussian_bump_forcing(3, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(3), nx, ny)
    P = sfde.Problem(0.7, 0.75, 1.0, 0.4, nx, ny, t, precision=prec)
    P.set_initial(psi)
    P.set_forcing(F)
    U = np.zeros((nt + 1, ny, nx))
    _, st = P.mgrit(U=U, m=4, max_levels=2, coarse=sfde.COARSE_BE, rel_tol=0.0, max_iter=1, check=False)
    res0 = st.residual_history()[0]
    U0 = np.zeros((nt + 1, ny, nx))
    U0[0] = psi
    _, nrm = gpu_residual(P, U0, 4)
    assert res0 == nrm or abs(res0 - nrm) <= 1e-15 * nrm, (res0, nrm)
    O = osfde.SFDE(0.7, 0.75, 1.0, 0.4, nx, ny, t)
    ref, scale = oracle_residual(O, U0, F)
    rn = np.sqrt(np.sum(ref ** 2))
    assert abs(res0 - rn) <= 2.0 ** (12 - 8 * 4) * scale + 2.0 ** -20 * rn
