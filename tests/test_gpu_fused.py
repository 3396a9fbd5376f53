"""One low-precision spectral step of the mixed-precision solver, fused (one kernel, four products
chained on chip) and as four tensor-core slice GEMMs, against the oracle's FP64 step.

Tolerances follow from the operand rounding: with unit roundoff u (2^-9 for BF16, 2^-11 for TF32),
the input, the four fixed matrices, the three intermediates and the output are each rounded once,
about nine independent relative perturbations of size <= u, so the relative Frobenius error of a
slice is about 2u; the bound is 5u.  The fused kernel and the chain round the same quantities and
differ only in the order of FP32 accumulation (and the modal factor's reciprocal), so they agree to
well below one rounding: relative Frobenius <= u/2, elementwise <= 4u of the slice maximum.
"""
import ctypes

import numpy as np
import pytest

from oracle import sfde as osfde
from sfde_workloads import sine_mode_amplitudes, sine_mode_nodal, time_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_06688_gb300 as sfde  # noqa: E402

PD = ctypes.POINTER(ctypes.c_double)


def lp_step(P, fused, scheme, U, n0, g=None, ut=None):
    L = sfde.lib()
    L.sfde_debug_lp_step.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, PD]
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.zeros_like(U)
    n2 = ctypes.c_double(-1.0)
    st = L.sfde_debug_lp_step(P.ctx, fused, scheme, U.ctypes.data, U.shape[0], n0,
                              None if g is None else np.ascontiguousarray(g).ctypes.data,
                              None if ut is None else np.ascontiguousarray(ut).ctypes.data,
                              out.ctypes.data, ctypes.byref(n2))
    return st, out, n2.value


def oracle_step(O, scheme, U, n0, g=None, ut=None):
    out = []
    for b in range(U.shape[0]):
        n = n0 + b
        dt = O.t[n] - O.t[n - 1]
        if scheme == 0:
            x = O.propagate(U[b], dt, "cn")
        elif scheme == 1:
            x = O.propagate(U[b], dt, "be")
        else:
            x = O.solve_S_fdm(U[b], 0.5 * dt)
        if g is not None:
            x = x + g[b]
        if ut is not None:
            x = x - ut[b]
        out.append(x)
    return np.stack(out)


def rel_fro(a, b):
    return np.sqrt(np.sum((a - b) ** 2, axis=(1, 2)) / np.sum(b ** 2, axis=(1, 2)))


CASES = [(255, 255, 160, 30), (200, 230, 6, 1), (100, 127, 40, 3)]


@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("nx,ny,batch,n0", CASES)
def test_fused_step_matches_chain_and_oracle(scheme, nx, ny, batch, n0):
    nt = n0 + batch + 3
    t = time_grid(nt, 1.0, "graded")
    O = osfde.SFDE(0.7, 0.8, 1.0, 0.5, nx, ny, t)
    P = sfde.Problem(0.7, 0.8, 1.0, 0.5, nx, ny, t, precision=sfde.PREC_MIXED_BF16)
    rng = np.random.default_rng(nx * 7 + scheme)
    U = rng.standard_normal((batch, ny, nx))
    ref = oracle_step(O, scheme, U, n0)
    st_f, xf, _ = lp_step(P, 1, scheme, U, n0)
    st_c, xc, _ = lp_step(P, 0, scheme, U, n0)
    assert st_f == 0 and st_c == 0, (sfde.sfde_strerror(st_f), sfde.sfde_strerror(st_c))
    u = 2.0 ** -9
    assert rel_fro(xf, ref).max() <= 5 * u, rel_fro(xf, ref).max()
    assert rel_fro(xc, ref).max() <= 5 * u, rel_fro(xc, ref).max()
    assert rel_fro(xf, xc).max() <= u / 2, rel_fro(xf, xc).max()
    scale = np.abs(xc).max(axis=(1, 2), keepdims=True)
    assert np.all(np.abs(xf - xc) <= 4 * u * scale)


@pytest.mark.parametrize("nx,ny,batch,n0", CASES[:1] + CASES[2:])
def test_fused_step_with_rhs_and_residual(nx, ny, batch, n0):
    """The residual form of Algorithm 1: Phi(u) + g - u_target, and its FP64 sum of squares."""
    nt = n0 + batch
    t = time_grid(nt, 2.0, "uniform")
    O = osfde.SFDE(0.6, 0.9, 1.5, 0.7, nx, ny, t)
    P = sfde.Problem(0.6, 0.9, 1.5, 0.7, nx, ny, t, precision=sfde.PREC_MIXED_BF16)
    rng = np.random.default_rng(nx + ny)
    U = rng.standard_normal((batch, ny, nx))
    g = 0.3 * rng.standard_normal((batch, ny, nx))
    ref0 = oracle_step(O, 0, U, n0, g)
    ut = ref0 + 0.05 * rng.standard_normal((batch, ny, nx))   # a near-solution: small differences
    ref = ref0 - ut
    for fused in (1, 0):
        st, x, n2 = lp_step(P, fused, 0, U, n0, g, ut)
        assert st == 0, sfde.sfde_strerror(st)
        # the difference is ~0.05 of the terms it is formed from: errors relative to the terms
        err = np.sqrt(np.sum((x - ref) ** 2, axis=(1, 2)) / np.sum(ref0 ** 2, axis=(1, 2)))
        assert err.max() <= 5 * 2.0 ** -9, err.max()
        assert abs(n2 - np.sum(x ** 2)) <= 2.0 ** -7 * np.sum(x ** 2)


def test_tf32_chain_step_and_fused_unsupported():
    nx = ny = 100
    t = time_grid(12, 1.0, "graded")
    O = osfde.SFDE(0.7, 0.8, 1.0, 0.5, nx, ny, t)
    P = sfde.Problem(0.7, 0.8, 1.0, 0.5, nx, ny, t, precision=sfde.PREC_MIXED_TF32)
    U = np.random.default_rng(3).standard_normal((5, ny, nx))
    st, _, _ = lp_step(P, 1, 0, U, 2)
    assert st == sfde.SFDE_EUNSUPPORTED
    st, x, _ = lp_step(P, 0, 0, U, 2)
    assert st == 0
    assert rel_fro(x, oracle_step(O, 0, U, 2)).max() <= 5 * 2.0 ** -11


def test_lp_step_argument_errors():
    t = time_grid(8, 1.0, "uniform")
    P = sfde.Problem(0.7, 0.8, 1.0, 0.5, 40, 40, t, precision=sfde.PREC_MIXED_BF16)
    U = np.zeros((4, 40, 40))
    assert lp_step(P, 0, 0, U, 6)[0] == sfde.SFDE_EINVAL      # n0 + batch - 1 > N_t
    assert lp_step(P, 0, 3, U, 1)[0] == sfde.SFDE_EINVAL      # unknown scheme
    assert lp_step(P, 1, 0, U, 1)[0] == sfde.SFDE_EUNSUPPORTED  # P = 64: no fused form
    Q = sfde.Problem(0.7, 0.8, 1.0, 0.5, 40, 40, t)
    assert lp_step(Q, 0, 0, U, 1)[0] == sfde.SFDE_EINVAL      # FP64 context


def test_mixed_bf16_solve_with_and_without_fused_step():
    """The whole mixed-precision solve reaches the FP64 answer either way (P = 128)."""
    nx, ny, nt = 100, 120, 128
    t = time_grid(nt, 1.0, "uniform")
    psi = sine_mode_nodal(sine_mode_amplitudes(5), nx, ny)
    O = osfde.SFDE(0.75, 0.85, 1.0, 1.0, nx, ny, t)
    ref = osfde.seq_timestep(O, psi)
    L = sfde.lib()
    L.sfde_debug_set_fused_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
    for fused in (1, 0):
        P = sfde.Problem(0.75, 0.85, 1.0, 1.0, nx, ny, t, precision=sfde.PREC_MIXED_BF16)
        P.set_initial(psi)
        assert L.sfde_debug_set_fused_step(P.ctx, fused) == 0
        U = np.zeros((nt + 1, ny, nx))
        _, stats = P.mgrit(U=U, m=4, max_levels=8, coarse=sfde.COARSE_BE, rel_tol=1e-11, max_iter=60)
        assert stats.converged
        assert np.abs(U - ref).max() <= 1e-8 * np.abs(ref).max(), fused


def mnorm(O, v):
    """||v||_{M_h} = (v, M_h v)^(1/2) with M_h = M_y (x) M_x (Sec. 2)."""
    return np.sqrt(np.sum(v * O.apply_mass(v)))


def lp_chain(P, mode, scheme, U, nchain, n0, g=None):
    L = sfde.lib()
    L.sfde_debug_lp_chain.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.zeros((U.shape[0], nchain) + U.shape[1:])
    st = L.sfde_debug_lp_chain(P.ctx, mode, scheme, U.ctypes.data, U.shape[0], nchain, n0,
                               None if g is None else np.ascontiguousarray(g).ctypes.data, out.ctypes.data)
    return st, out


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("nx,ny,batch,nchain", [(255, 255, 150, 2), (100, 127, 3, 3), (200, 180, 2, 15)])
def test_chained_steps(scheme, nx, ny, batch, nchain):
    """The F-relaxation chain of one fused launch (each CTA keeps its slice on chip from step to
    step) equals single fused launches bit for bit; it, the four-GEMM steps and the chain run in the
    step's eigenbasis (transforms, FP32 recurrence per mode, transforms back) all follow the
    oracle's FP64 steps.  Both propagators are contractions in the M_h-norm (Sec. 3: their modal
    factors are at most 1 in modulus), so rounding errors introduced at each step add up in that
    norm: after k + 1 steps at most 5u (k + 1).  The two low-precision paths agree to u/2 on the
    first step, from identical BF16 input; after it their inputs differ slightly and their
    roundings are no longer the same, so they are compared through the oracle."""
    n0 = 2
    nt = n0 + batch * nchain
    t = time_grid(nt, 1.0, "graded")
    O = osfde.SFDE(0.7, 0.8, 1.0, 0.5, nx, ny, t)
    P = sfde.Problem(0.7, 0.8, 1.0, 0.5, nx, ny, t, precision=sfde.PREC_MIXED_BF16)
    rng = np.random.default_rng(nx + nchain + scheme)
    U = rng.standard_normal((batch, ny, nx))
    g = 0.2 * rng.standard_normal((batch, nchain, ny, nx))
    st1, x1 = lp_chain(P, 1, scheme, U, nchain, n0, g)
    st2, x2 = lp_chain(P, 2, scheme, U, nchain, n0, g)
    st0, x0 = lp_chain(P, 0, scheme, U, nchain, n0, g)
    st3, x3 = lp_chain(P, 3, scheme, U, nchain, n0, g)
    assert st1 == 0 and st2 == 0 and st0 == 0 and st3 == 0
    assert np.array_equal(x1, x2)
    u = 2.0 ** -9
    for b in range(batch):
        x = U[b]
        for k in range(nchain):
            n = n0 + b * nchain + k
            x = O.propagate(x, O.t[n] - O.t[n - 1], "cn" if scheme == 0 else "be") + g[b, k]
            mref = mnorm(O, x)
            for xs in (x1, x0, x3):
                rel = mnorm(O, xs[b, k] - x) / mref
                assert rel <= 5 * u * (k + 1), (b, k, rel)
        d = np.sqrt(np.sum((x1[b, 0] - x0[b, 0]) ** 2) / np.sum(x0[b, 0] ** 2))
        assert d <= u / 2, (b, d)


def set_pair(P, mode):
    L = sfde.lib()
    L.sfde_debug_set_fused_pair.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert L.sfde_debug_set_fused_pair(P.ctx, mode) == 0


@pytest.mark.parametrize("nx,ny,batch,nchain", [(255, 255, 3, 1), (230, 200, 2, 7), (255, 240, 90, 2),
                                                (250, 255, 5, 3)])
def test_pair_forms_equal_one_cta(nx, ny, batch, nchain):
    """A CTA pair per slice (each CTA holding half the rows of every operand, the products issued
    over the pair) and a CTA pair per two slices (odd batches leave one pair a single slice) round
    exactly the same sums as one CTA per slice: the accumulation order of every output element is the
    same, so the results are identical, for the three step kinds, with right-hand side and target,
    and along chains (the sum of squares of a residual step, FP32 partial sums, to 2^-20)."""
    n0 = 1
    nt = n0 + batch * nchain + 1
    t = time_grid(nt, 1.0, "graded")
    P = sfde.Problem(0.65, 0.85, 1.3, 0.4, nx, ny, t, precision=sfde.PREC_MIXED_BF16)
    rng = np.random.default_rng(nx + ny + batch)
    U = rng.standard_normal((batch, ny, nx))
    g = 0.2 * rng.standard_normal((batch, nchain, ny, nx))
    res = {}
    for mode in (0, 2, 3):
        set_pair(P, mode)
        out = []
        if nchain == 1:
            for scheme in (0, 1, 2):
                st, x, _ = lp_step(P, 1, scheme, U, n0)
                assert st == 0, sfde.sfde_strerror(st)
                out.append(x)
            st, x, n2 = lp_step(P, 1, 0, U, n0, g[:, 0], 0.5 * U)
            assert st == 0, sfde.sfde_strerror(st)
            out += [x, np.array([n2])]
        else:
            for scheme in (0, 1):
                st, x = lp_chain(P, 1, scheme, U, nchain, n0, g)
                assert st == 0, sfde.sfde_strerror(st)
                out.append(x)
        res[mode] = out
    for mode in (2, 3):
        for a, b in zip(res[0], res[mode]):
            if a.shape == (1,):   # the sum of squares: FP32 partial sums, taken in another order
                assert abs(a[0] - b[0]) <= 2.0 ** -20 * abs(a[0]), (mode, a, b)
            else:
                assert np.array_equal(a, b), (mode, np.abs(a - b).max())


def test_mixed_bf16_solve_pair_forms():
    """A whole mixed-precision solve at P = 256 with every fused step on a CTA pair per slice, or per
    two slices, reaches the FP64 answer, as with one CTA per slice."""
    nx, ny, nt = 255, 255, 64
    t = time_grid(nt, 1.0, "uniform")
    psi = sine_mode_nodal(sine_mode_amplitudes(4), nx, ny)
    O = osfde.SFDE(0.6, 0.9, 1.0, 0.5, nx, ny, t)
    ref = osfde.seq_timestep(O, psi)
    for mode in (2, 3, 0):
        P = sfde.Problem(0.6, 0.9, 1.0, 0.5, nx, ny, t, precision=sfde.PREC_MIXED_BF16)
        P.set_initial(psi)
        set_pair(P, mode)
        U = np.zeros((nt + 1, ny, nx))
        _, stats = P.mgrit(U=U, m=8, max_levels=4, coarse=sfde.COARSE_BE, rel_tol=1e-10, max_iter=60)
        assert stats.converged
        assert np.abs(U - ref).max() <= 1e-8 * np.abs(ref).max(), mode


@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("nx,ny,batch,n0", CASES)
def test_step_elementwise_error_bound_against_oracle(scheme, nx, ny, batch, n0):
    """Element by element against the oracle's FP64 step.  The low-precision step computes
    X = V_y [f o (L_y^T U L_x)] V_x^T (L = W = M V for a propagator, L = V for the solve, f the modal
    factor of Eq. (3.7)) with the input, four matrices, three intermediates and the output each
    rounded to BF16 (unit roundoff u = 2^-9) and FP32 accumulation; to first order every element's
    error is at most 9 u times the same chain taken in absolute values,
        B = |V_y| (|f| o (|L_y|^T |U| |L_x|)) |V_x|^T,
    so |x - x_oracle| <= 10 u B holds element by element, for the fused kernel and the chain."""
    nt = n0 + batch + 3
    t = time_grid(nt, 1.0, "graded")
    O = osfde.SFDE(0.7, 0.8, 1.0, 0.5, nx, ny, t)
    P = sfde.Problem(0.7, 0.8, 1.0, 0.5, nx, ny, t, precision=sfde.PREC_MIXED_BF16)
    rng = np.random.default_rng(nx * 11 + scheme)
    U = rng.standard_normal((batch, ny, nx))
    ref = oracle_step(O, scheme, U, n0)
    lx, Vx, ly, Vy = O.eig()
    sig = O.sigma()
    Lx, Ly = (O.Mx @ Vx, O.My @ Vy) if scheme < 2 else (Vx, Vy)
    aVx, aVy, aLx, aLy = np.abs(Vx), np.abs(Vy), np.abs(Lx), np.abs(Ly)
    u = 2.0 ** -9
    for fused in (1, 0):
        st, x, _ = lp_step(P, fused, scheme, U, n0)
        assert st == 0, sfde.sfde_strerror(st)
        worst = 0.0
        for b in range(batch):
            dt = O.t[n0 + b] - O.t[n0 + b - 1]
            f = (osfde.modal_lambda(sig, dt, "cn") if scheme == 0 else
                 osfde.modal_lambda(sig, dt, "be") if scheme == 1 else 1.0 / (1.0 + 0.5 * dt * sig))
            B = aVy @ (np.abs(f) * (aLy.T @ np.abs(U[b]) @ aLx)) @ aVx.T
            r = np.abs(x[b] - ref[b]) / (u * B)
            worst = max(worst, float(r.max()))
        assert worst <= 10.0, (fused, worst)


@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("nx,ny,batch,n0", [(255, 255, 40, 30), (200, 230, 6, 1), (511, 300, 5, 2)])
def test_fp32_step_elementwise_error_bound(scheme, nx, ny, batch, n0):
    """The FP32 form's step (four slice GEMMs, each product from three TF32 products, FP32
    intermediates) element by element against the oracle: the same first-order bound as for BF16 with
    the unit roundoff of the FP32 products, u = 2^-20 (the dropped lo x lo term and the low parts read
    as TF32), |x - x_oracle| <= 10 u B."""
    nt = n0 + batch + 3
    t = time_grid(nt, 1.0, "graded")
    O = osfde.SFDE(0.7, 0.8, 1.0, 0.5, nx, ny, t)
    P = sfde.Problem(0.7, 0.8, 1.0, 0.5, nx, ny, t, precision=sfde.PREC_MIXED_FP32)
    rng = np.random.default_rng(nx * 13 + scheme)
    U = rng.standard_normal((batch, ny, nx))
    ref = oracle_step(O, scheme, U, n0)
    st, x, _ = lp_step(P, 0, scheme, U, n0)
    assert st == 0, sfde.sfde_strerror(st)
    lx, Vx, ly, Vy = O.eig()
    sig = O.sigma()
    Lx, Ly = (O.Mx @ Vx, O.My @ Vy) if scheme < 2 else (Vx, Vy)
    u = 2.0 ** -20
    worst = 0.0
    for b in range(batch):
        dt = O.t[n0 + b] - O.t[n0 + b - 1]
        f = (osfde.modal_lambda(sig, dt, "cn") if scheme == 0 else
             osfde.modal_lambda(sig, dt, "be") if scheme == 1 else 1.0 / (1.0 + 0.5 * dt * sig))
        B = np.abs(Vy) @ (np.abs(f) * (np.abs(Ly).T @ np.abs(U[b]) @ np.abs(Lx))) @ np.abs(Vx).T
        worst = max(worst, float((np.abs(x[b] - ref[b]) / (u * B)).max()))
    assert worst <= 10.0, worst
    # and far below the TF32 form's error
    assert rel_fro(x, ref).max() <= 2.0 ** -16, rel_fro(x, ref).max()
