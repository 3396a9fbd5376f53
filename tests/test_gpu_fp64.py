"""GPU parity of the FP64 path against the FP64 CPU oracle, through the C ABI.

Tolerances: the FP64 path and the oracle evaluate the same algebra in a different order
(series vs 40-digit coefficients, Jacobi vs LAPACK eigenpairs, tiled vs BLAS products), so
results agree to a small multiple of cond * eps; 1e-11 relative (max norm) is used for fields,
1e-12 for coefficients.  The MGRIT target in FP64 is 1e-10 relative to the oracle.
"""
import numpy as np
import pytest

from oracle import mgrit as omgrit
from oracle import sfde as osfde
from sfde_workloads import (WORKLOADS, gaussian_bump_forcing, sine_mode_amplitudes,
                            sine_mode_nodal, time_grid)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_06688_gb300 as sfde  # noqa: E402


def relerr(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def make(beta, gamma, kx, ky, nx, ny, t, omega=(0.0, 1.0, 0.0, 1.0), forcing=None, psi0=None):
    P = sfde.Problem(beta, gamma, kx, ky, nx, ny, t, omega)
    if psi0 is not None:
        P.set_initial(np.ascontiguousarray(psi0))
    P.set_forcing(forcing)
    O = osfde.SFDE(beta, gamma, kx, ky, nx, ny, t, omega)
    return P, O


@pytest.mark.parametrize("n,rho", [(31, 0.75), (255, 0.6), (1023, 0.55), (1, 0.9), (100, 0.99)])
def test_toeplitz_coefficients(n, rho):
    P = sfde.Problem(rho, 0.8, 1.0, 1.0, n, 3, time_grid(2))
    a, _, _ = P.operator(0)
    ref = osfde.riesz_coefficients(n, rho)
    assert np.all(np.abs(a - ref) <= 1e-12 * np.abs(ref) + 1e-15 * abs(ref[0]))


@pytest.mark.parametrize("n,rho", [(31, 0.75), (200, 0.6), (511, 0.95)])
def test_generalised_eigenpairs(n, rho):
    P = sfde.Problem(rho, 0.8, 1.0, 1.0, n, 3, time_grid(2))
    _, lam, V = P.operator(0)
    A, M = osfde.stiffness_1d(n, rho), osfde.mass_1d(n)
    ref = np.sort(np.linalg.eigvalsh(np.linalg.solve(np.linalg.cholesky(M), np.linalg.solve(np.linalg.cholesky(M), A).T)))
    assert relerr(np.sort(lam), ref) < 1e-12
    assert np.abs(V.T @ M @ V - np.eye(n)).max() < 1e-12
    assert np.abs(A @ V - M @ V * lam[None, :]).max() < 1e-11 * lam.max() * np.abs(M @ V).max()


@pytest.mark.parametrize("nx,ny,grid", [(5, 7, "uniform"), (50, 70, "graded"), (63, 33, "uniform"), (129, 64, "graded")])
def test_step_batch_matches_oracle(nx, ny, grid):
    t = time_grid(24, 1.0, grid)
    F, _ = gaussian_bump_forcing(3, nx, ny, t)
    P, O = make(0.7, 0.85, 1.3, 0.4, nx, ny, t, forcing=F)
    rng = np.random.default_rng(0)
    batch, n0, dn = 6, 2, 4
    src = rng.standard_normal((batch, ny, nx))
    dst = np.zeros_like(src)
    P.step_batch(n0, dn, src, dst)
    for b in range(batch):
        n = n0 + b * dn
        ref = O.step(src[b], n, F.dense(n))
        assert relerr(dst[b], ref) < 1e-11, (b, relerr(dst[b], ref))


def test_step_batch_device_tensors():
    t = time_grid(8)
    P, O = make(0.6, 0.9, 1.0, 0.5, 40, 24, t)
    src = torch.randn(3, 24, 40, dtype=torch.float64, device="cuda")
    dst = torch.empty_like(src)
    P.step_batch(1, 1, src, dst)
    s = src.cpu().numpy()
    for b in range(3):
        assert relerr(dst[b].cpu().numpy(), O.step(s[b], 1 + b)) < 1e-11


@pytest.mark.parametrize("nx,ny,nt,grid", [(31, 31, 64, "uniform"), (20, 45, 37, "graded"), (1, 6, 5, "uniform")])
def test_seq_timestep_matches_oracle(nx, ny, nt, grid):
    t = time_grid(nt, 1.0, grid)
    F, _ = gaussian_bump_forcing(9, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(2), nx, ny)
    P, O = make(0.65, 0.8, 0.7, 1.9, nx, ny, t, forcing=F, psi0=psi)
    U = np.zeros((nt + 1, ny, nx))
    UT = np.zeros((ny, nx))
    P.seq(U, UT)
    ref = osfde.seq_timestep(O, psi, F)
    assert relerr(U, ref) < 1e-11
    assert np.array_equal(UT, U[-1])


def test_manufactured_two_level_matches_oracle():
    w = WORKLOADS["manufactured_N31_Nt64"]
    t = w.t()
    P, O = make(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t, forcing=w.forcing(), psi0=w.initial())
    for coarse, cname in ((sfde.COARSE_BE, "be"), (sfde.COARSE_CN, "cn")):
        U = np.zeros((w.nt + 1, w.ny, w.nx))
        _, st = P.mgrit(U=U, m=w.m, max_levels=2, coarse=coarse, rel_tol=1e-10)
        ref = omgrit.mgrit(O, w.initial(), w.forcing(), m=w.m, max_levels=2, coarse=cname, rel_tol=1e-10)
        assert st.converged and st.iters == ref.iters and st.levels == 2
        h = st.residual_history()
        for a, b in zip(h, ref.history):
            assert abs(a - b) <= 1e-9 * ref.history[0]
        assert relerr(U, ref.U) < 1e-11


@pytest.mark.parametrize("relax", ["FCF", "F"])
@pytest.mark.parametrize("coarse", ["cn", "be"])
def test_multilevel_graded_random_init_matches_oracle(relax, coarse):
    nx, ny, nt, m = 20, 13, 64, 4
    t = time_grid(nt, 1.0, "graded")
    F, _ = gaussian_bump_forcing(5, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(4), nx, ny)
    P, O = make(0.6, 0.9, 1.0, 0.5, nx, ny, t, forcing=F, psi0=psi)
    U = np.zeros((nt + 1, ny, nx))
    _, st = P.mgrit(U=U, m=m, max_levels=3, coarse={"cn": sfde.COARSE_CN, "be": sfde.COARSE_BE}[coarse],
                    relax={"FCF": sfde.RELAX_FCF, "F": sfde.RELAX_F}[relax], rel_tol=1e-11, max_iter=60,
                    init_seed=12345, check=False)
    ref = omgrit.mgrit(O, psi, F, m=m, max_levels=3, coarse=coarse, relax=relax, rel_tol=1e-11,
                       max_iter=60, init_seed=12345)
    assert st.levels == ref.levels == 3
    assert st.iters == ref.iters
    h = st.residual_history()
    for a, b in zip(h, ref.history):
        assert abs(a - b) <= 1e-9 * ref.history[0]
    assert relerr(U, ref.U) < 1e-10


def test_sine_N255_Nt1024_full_size():
    """The benchmarked workload at full size in the launch configuration bench.py times: GPU
    FP64 MGRIT against the oracle's modal execution of the same iteration (same iterates up to
    rounding) and against the exact sequential solution at sampled time points."""
    w = WORKLOADS["sine_N255_Nt1024"]
    t = w.t()
    psi = w.initial()
    P, O = make(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, t, psi0=psi)
    U = torch.zeros((w.nt + 1, w.ny, w.nx), dtype=torch.float64, device="cuda")
    _, st = P.mgrit(U=U, m=w.m, max_levels=32, coarse=sfde.COARSE_AUTO, rel_tol=w.rel_tol, max_iter=200)
    assert st.converged and st.levels == 4
    ref = omgrit.mgrit_modal(O, psi, None, m=w.m, max_levels=32, coarse="be" if st.coarse_used == 1 else "cn",
                             rel_tol=w.rel_tol, max_iter=200)
    assert st.iters == ref.iters
    h = st.residual_history()
    for a, b in zip(h, ref.history):
        assert abs(a - b) <= 1e-8 * ref.history[0]
    # errors relative to the max norm of the space-time solution (u decays by ~1e-7 up to T)
    scale = np.abs(psi).max()
    UT = U[-1].cpu().numpy()
    assert np.abs(UT - ref.U).max() < 1e-10 * scale
    exact = osfde.spectral_sequential(O, psi, None, keep=[128, 512, 1024])
    for n in (128, 512, 1024):
        assert np.abs(U[n].cpu().numpy() - exact[n]).max() < 1e-8 * scale


def test_edge_cases_and_errors():
    t = time_grid(1)
    P, O = make(0.8, 0.7, 1.0, 1.0, 3, 4, t, psi0=np.ones((4, 3)))
    U = np.zeros((2, 4, 3))
    _, st = P.mgrit(U=U, m=2)       # a single step: one level, sequential
    assert st.levels == 1
    assert relerr(U[1], O.step(np.ones((4, 3)), 1)) < 1e-12
    # max_iter reached -> ENOCONV with stats filled
    t = time_grid(64)
    P, _ = make(0.6, 0.9, 1.0, 0.5, 16, 16, t, psi0=sine_mode_nodal(sine_mode_amplitudes(1), 16, 16))
    st_code, st = P.mgrit(m=4, max_iter=2, rel_tol=1e-14, coarse=sfde.COARSE_BE, check=False)
    assert st_code == sfde.SFDE_ENOCONV and st.iters == 2 and not st.converged
    # non-finite initial data -> ENOCONV
    bad = np.full((16, 16), np.nan)
    P.set_initial(bad)
    st_code, st = P.mgrit(m=4, max_iter=5, check=False)
    assert st_code == sfde.SFDE_ENOCONV
    # step index out of range
    with pytest.raises(sfde.SfdeError):
        P.step_batch(64, 1, np.zeros((2, 16, 16)), np.zeros((2, 16, 16)))


@pytest.mark.parametrize("stop", ["cpoint", "sform"])
@pytest.mark.parametrize("skip", [False, True])
def test_skip_first_down_and_space_time_stop_match_oracle(skip, stop):
    """The skip-first-down option (Sec. 3.2) and the space-time (S-form) stopping test against the
    oracle's Algorithm 1 with the same options: same iteration count, residual history and iterate.
    The GPU evaluates the S-form norm after a relaxation at the C-points only (rho_km = S_km r_k,
    the F-point rows being satisfied); the oracle sums the full space-time residual."""
    nx, ny, nt, m = 20, 13, 64, 4
    t = time_grid(nt, 1.0, "graded")
    F, _ = gaussian_bump_forcing(5, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(4), nx, ny)
    P, O = make(0.6, 0.9, 1.0, 0.5, nx, ny, t, forcing=F, psi0=psi)
    U = np.zeros((nt + 1, ny, nx))
    _, st = P.mgrit(U=U, m=m, max_levels=3, coarse=sfde.COARSE_BE, rel_tol=1e-11, max_iter=60,
                    skip_first_down=skip, stop_kind=sfde.STOP_SFORM if stop == "sform" else sfde.STOP_NATIVE)
    ref = omgrit.mgrit(O, psi, F, m=m, max_levels=3, coarse="be", rel_tol=1e-11, max_iter=60,
                       skip_first_down=skip, stop=stop)
    assert st.converged and ref.converged
    assert st.iters == ref.iters, (st.iters, ref.iters)
    h = st.residual_history()
    top = max(ref.history)
    for k, (a, b) in enumerate(zip(h, ref.history)):
        assert abs(a - b) <= 1e-9 * top, (k, a, b)
    assert relerr(U, ref.U) < 1e-10
    if stop == "sform":
        # the reference norm is the initial guess's space-time residual
        rho0 = omgrit.space_time_residual(O, omgrit.initial_guess(psi, nt), F)
        assert abs(st.res0 - np.sqrt((rho0 ** 2).sum())) <= 1e-12 * st.res0


def test_options_validation():
    P, _ = make(0.6, 0.9, 1.0, 0.5, 8, 8, time_grid(16))
    for kw in (dict(skip_first_down=2), dict(stop_kind=2), dict(stop_kind=-1)):
        opts = sfde.make_opts(m=4, **{k: 0 for k in kw})
        for k, v in kw.items():
            setattr(opts, k, v)
        st = sfde.lib().mgrit_solve(P.ctx, sfde._binding.C.byref(opts), None, None, None)
        assert st == sfde.SFDE_EINVAL, kw


def test_dense_forcing_matches_oracle():
    """sfde_set_forcing_dense (a non-separable load, a bump moving in x): the single step, sequential
    stepping and FP64 MGRIT against the oracle with the same load; clearing and replacing the load."""
    from sfde_workloads import moving_bump_dense_forcing
    nx, ny, nt = 40, 33, 24
    t = time_grid(nt, 1.0, "graded")
    D, _ = moving_bump_dense_forcing(7, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(3), nx, ny)
    P, O = make(0.7, 0.85, 1.3, 0.4, nx, ny, t, psi0=psi)
    P.set_forcing_dense(torch.from_numpy(D.F).cuda())
    rng = np.random.default_rng(1)
    src = rng.standard_normal((5, ny, nx))
    dst = np.zeros_like(src)
    P.step_batch(2, 4, src, dst)
    for b in range(5):
        n = 2 + 4 * b
        assert relerr(dst[b], O.step(src[b], n, D.dense(n))) < 1e-11, b
    U = np.zeros((nt + 1, ny, nx))
    P.seq(U)
    ref = osfde.seq_timestep(O, psi, D)
    assert relerr(U, ref) < 1e-11
    U[:] = 0
    _, st = P.mgrit(U=U, m=4, max_levels=3, coarse=sfde.COARSE_BE, rel_tol=1e-11, max_iter=60)
    r = omgrit.mgrit(O, psi, D, m=4, max_levels=3, coarse="be", rel_tol=1e-11, max_iter=60)
    assert st.iters == r.iters and relerr(U, r.U) < 1e-10
    # cleared: no load
    P.set_forcing_dense(None)
    P.seq(U)
    assert relerr(U, osfde.seq_timestep(O, psi)) < 1e-11
    # a separable load replaces a dense one, and a dense one a separable one
    F, _ = gaussian_bump_forcing(2, nx, ny, t)
    P.set_forcing_dense(D.F)
    P.set_forcing(F)
    P.seq(U)
    assert relerr(U, osfde.seq_timestep(O, psi, F)) < 1e-11
    P.set_forcing_dense(D.F)
    P.seq(U)
    assert relerr(U, ref) < 1e-11
    with pytest.raises(ValueError):
        P.set_forcing_dense(D.F[:-1])


@pytest.mark.parametrize("relax,levels,m", [("FCF", 3, 4), ("F", 2, 4), ("FCF", 2, 2)])
def test_shishkin_grid_matches_oracle(relax, levels, m):
    """The piecewise-uniform partition of Sec. 4.1 (N/4 steps on [0, s], N/2 on [s, T - s], N/4 on
    [T - s, T], s = 2 eps ln N), with MGRIT (FCF) and the parareal form (F-relaxation, two levels):
    the GPU iteration against the oracle's, iteration by iteration, and its fixed point against
    sequential stepping."""
    nx, ny, nt = 24, 17, 64
    t = time_grid(nt, 1.0, "shishkin", eps=2.0 ** -6)
    assert len(set(np.round(np.diff(t), 15))) >= 2          # really piecewise uniform
    F, _ = gaussian_bump_forcing(8, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(6), nx, ny)
    P, O = make(0.6, 0.7, 3.0, 7.5, nx, ny, t, forcing=F, psi0=psi)
    U = np.zeros((nt + 1, ny, nx))
    _, st = P.mgrit(U=U, m=m, max_levels=levels, coarse=sfde.COARSE_BE,
                    relax={"FCF": sfde.RELAX_FCF, "F": sfde.RELAX_F}[relax], rel_tol=1e-11, max_iter=80)
    ref = omgrit.mgrit(O, psi, F, m=m, max_levels=levels, coarse="be", relax=relax, rel_tol=1e-11, max_iter=80)
    assert st.converged and st.iters == ref.iters and st.levels == ref.levels == levels
    for a, b in zip(st.residual_history(), ref.history):
        assert abs(a - b) <= 1e-9 * ref.history[0]
    assert relerr(U, ref.U) < 1e-10
    assert relerr(U, osfde.seq_timestep(O, psi, F)) < 1e-9


@pytest.mark.parametrize("grid", ["uniform", "graded", "shishkin"])
def test_two_level_bound_on_device_matches_oracle(grid):
    """Theorem 3.1's bound (Eq. (3.11)) evaluated on the device over every mode equals the oracle's
    evaluation over every step size, for several m and both coarse propagators."""
    from oracle import analysis
    nt = 64
    t = time_grid(nt, 1.0, grid, eps=2.0 ** -6 if grid == "shishkin" else None)
    P, O = make(0.7, 0.85, 1.3, 0.6, 47, 33, t)
    for m in (2, 4, 8, 16):
        for coarse, name in ((sfde.COARSE_CN, "cn"), (sfde.COARSE_BE, "be")):
            got = P.two_level_bound(m, coarse)
            ref = analysis.tub_bound(O.sigma(), t, m, name)
            assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (m, name, got, ref)
    with pytest.raises(sfde.SfdeError):
        P.two_level_bound(3)            # 3 does not divide 64


def test_coarsening_factor_chosen_by_the_two_level_analysis():
    """mgrit_opts.m = 0: the coarsening factor is the argmin over m in {2, 4, 8, 16, 32} of
    ceil(log tol / log b(m)) * 2 m / (m - 1), b(m) the bound of the coarse propagator in use (AUTO: CN
    where its bound is below 1), computed here from the oracle's bounds; the solve with m = 0 uses it
    and still reaches the oracle's sequential solution."""
    import math
    from oracle import analysis
    nx, ny, nt = 24, 20, 128
    t = time_grid(nt)
    F, _ = gaussian_bump_forcing(3, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(2), nx, ny)
    for beta, gamma, kx, ky in ((0.7, 0.8, 1.0, 1.0), (0.6, 0.9, 0.05, 0.02)):
        P, O = make(beta, gamma, kx, ky, nx, ny, t, forcing=F, psi0=psi)
        tol = 1e-10
        best, best_cost = None, math.inf
        for m in (2, 4, 8, 16, 32):
            bcn = analysis.tub_bound(O.sigma(), t, m, "cn")
            b = bcn if bcn < 1.0 else analysis.tub_bound(O.sigma(), t, m, "be")
            if not b < 1.0:
                continue
            cost = max(1.0, math.ceil(math.log(tol) / math.log(b))) * 2.0 * m / (m - 1)
            if cost <= best_cost:
                best, best_cost = m, cost
        assert P.choose_coarsening(sfde.COARSE_AUTO, tol) == best, (beta, gamma, kx, ky)
        U = np.zeros((nt + 1, ny, nx))
        _, st = P.mgrit(U=U, m=0, max_levels=32, coarse=sfde.COARSE_AUTO, rel_tol=tol, max_iter=100)
        assert st.converged and st.m_used == best
        assert relerr(U, osfde.seq_timestep(O, psi, F)) < 1e-9


def test_propagate_batch_matches_oracle():
    """sfde_propagate_batch: the coarse propagators (Eq. (3.4) and the backward-Euler one) with their
    own step sizes and a right-hand side, against the oracle."""
    nx, ny = 40, 27
    t = time_grid(8)
    P, O = make(0.65, 0.9, 1.2, 0.3, nx, ny, t)
    rng = np.random.default_rng(9)
    V, G = rng.standard_normal((3, ny, nx)), rng.standard_normal((3, ny, nx))
    dts = np.array([0.01, 0.5, 2.0])
    for scheme, name in ((sfde.COARSE_CN, "cn"), (sfde.COARSE_BE, "be")):
        out = np.zeros_like(V)
        sfde.sfde_propagate_batch(P.ctx, scheme, dts, V, out, G)
        for b in range(3):
            assert relerr(out[b], O.propagate(V[b], dts[b], name) + G[b]) < 1e-11, (name, b)
        sfde.sfde_propagate_batch(P.ctx, scheme, dts, V, out)
        assert relerr(out[1], O.propagate(V[1], dts[1], name)) < 1e-11
    with pytest.raises(sfde.SfdeError):
        sfde.sfde_propagate_batch(P.ctx, sfde.COARSE_BE, np.array([0.1, -1.0, 0.1]), V, np.zeros_like(V))


def test_time_sharded_driver_with_library_steps_matches_mgrit_solve():
    """The time-sharded driver on one rank with the library's steps (sfde_step_batch for the fine
    level, sfde_propagate_batch for the coarse ones) reproduces mgrit_solve's FP64 iteration."""
    from paper_1805_06688_gb300.timeshard import LibraryStepper, time_sharded_mgrit
    nx, ny, nt, m = 30, 22, 64, 4
    t = time_grid(nt, 1.0, "graded")
    F, _ = gaussian_bump_forcing(4, nx, ny, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(7), nx, ny)
    P, O = make(0.6, 0.9, 1.0, 0.5, nx, ny, t, forcing=F, psi0=psi)
    U = np.zeros((nt + 1, ny, nx))
    _, st = P.mgrit(U=U, m=m, max_levels=3, coarse=sfde.COARSE_BE, rel_tol=1e-11, max_iter=60)
    res = time_sharded_mgrit(LibraryStepper(P, sfde.COARSE_BE), t, torch.from_numpy(psi).cuda(), m, max_levels=3,
                             rel_tol=1e-11, max_iter=60)
    assert res.converged and res.iters == st.iters and res.lo == 0 and res.hi == nt
    for a, b in zip(res.history, st.residual_history()):
        assert abs(a - b) <= 1e-10 * st.res0
    assert relerr(res.U.cpu().numpy(), U) < 1e-11
