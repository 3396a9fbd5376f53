"""Pins of the oracle's MGRIT (Algorithm 1, Lemma 3.1, Theorem 3.1, Table 5)."""
import json
import os

import numpy as np
import pytest

from oracle import analysis, mgrit, sfde
from oracle.mgrit import splitmix64_uniform
from sfde_workloads import (gaussian_bump_forcing, manufactured_forcing, manufactured_initial,
                            sine_mode_amplitudes, sine_mode_nodal, time_grid)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def test_splitmix64_published_sequence():
    """SplitMix64 seeded with 0 starts 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f."""
    ref = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    want = np.array([(v >> 11) * 2.0 ** -53 * 2 - 1 for v in ref])
    np.testing.assert_array_equal(splitmix64_uniform(0, 0, 3), want)


def _small(nt=32, grid="uniform", nx=5, ny=4, beta=0.7, gamma=0.85, kx=1.0, ky=0.6):
    t = time_grid(nt, 1.0, grid)
    P = sfde.SFDE(beta, gamma, kx, ky, nx, ny, t)
    U0 = sine_mode_nodal(sine_mode_amplitudes(5), nx, ny)
    F, _ = gaussian_bump_forcing(6, nx, ny, t)
    return P, U0, F


@pytest.mark.parametrize("coarse", ["cn", "be"])
@pytest.mark.parametrize("grid,m,levels", [("uniform", 2, 32), ("graded", 4, 2), ("uniform", 4, 3)])
def test_fixed_point_is_sequential_solution(coarse, grid, m, levels):
    """The MGRIT fixed point is the solution of Eq. (3.1), i.e. sequential stepping."""
    P, U0, F = _small(grid=grid)
    seq = sfde.seq_timestep(P, U0, F, dense=True)
    r = mgrit.mgrit(P, U0, F, m=m, max_levels=levels, coarse=coarse, rel_tol=1e-13, max_iter=60,
                    dense=True, init_seed=7)
    assert r.converged
    assert np.abs(r.U - seq).max() <= 1e-11 * np.abs(seq).max()


@pytest.mark.parametrize("coarse", ["cn", "be"])
def test_nodal_and_modal_mgrit_agree(coarse):
    P, U0, F = _small(nt=64, grid="graded", nx=6, ny=7)
    a = mgrit.mgrit(P, U0, F, m=4, coarse=coarse, rel_tol=1e-12, max_iter=30, init_seed=3)
    b = mgrit.mgrit_modal(P, U0, F, m=4, coarse=coarse, rel_tol=1e-12, max_iter=30, init_seed=3,
                          keep_all=True)
    assert a.iters == b.iters and a.levels == b.levels == 3
    h0 = a.history[0]
    for x, y in zip(a.history, b.history):
        assert abs(x - y) <= 1e-11 * h0
    assert np.abs(a.U - b.U).max() <= 1e-12 * np.abs(a.U).max()


def test_lemma_3_1_two_level_propagator():
    """One two-level FCF iteration leaves the C-point error of Lemma 3.1 (time-dependent Psi_n)."""
    nt, m = 16, 4
    P, U0, F = _small(nt=nt, grid="graded", nx=3, ny=4)
    seq = sfde.seq_timestep(P, U0, F, dense=True)
    u0 = mgrit.initial_guess(U0, nt, init_seed=11)
    E_c = [seq[k * m] - u0[k * m] for k in range(nt // m + 1)]
    for coarse in ("cn", "be"):
        r = mgrit.mgrit(P, U0, F, m=m, max_levels=2, coarse=coarse, rel_tol=0.0, max_iter=1,
                        init_seed=11, dense=True)
        pred = analysis.lemma31_cpoint_error(P, E_c, m, coarse)
        for k in range(nt // m + 1):
            got = seq[k * m] - r.U[k * m]
            assert np.abs(got - pred[k]).max() <= 1e-12 * np.abs(seq).max(), (coarse, k)
        assert np.abs(seq[m] - r.U[m]).max() <= 1e-13 * np.abs(seq).max()  # E~_m = 0


def test_two_level_is_exact_after_finitely_many_iterations():
    """Two-level FCF with N_c coarse intervals reproduces sequential stepping exactly after at
    most N_c/2 + 1 iterations (each iteration makes two more C-points exact, Lemma 3.1)."""
    P, U0, F = _small(nt=32)
    seq = sfde.seq_timestep(P, U0, F)
    r = mgrit.mgrit(P, U0, F, m=4, max_levels=2, coarse="cn", rel_tol=0.0, max_iter=5)
    assert np.abs(r.U - seq).max() <= 1e-13 * np.abs(seq).max()


@pytest.mark.parametrize("m,key", [(2, "m2"), (16, "m16")])
def test_table5_convergence_factor_magnitude(m, key):
    """Example 4.2, Table 5 setting (M = 16, N = 256, beta = 0.6, gamma = 0.7, K_x = 2, K_y = 0.5):
    the measured two-level factor is of the printed magnitude (printed values are for P1
    triangles) and below Theorem 3.1's bound evaluated on this operator's spectrum."""
    tab = json.load(open(GOLDEN))["table5"]
    n, nt = tab["M"] - 1, tab["N"]
    t = time_grid(nt)
    P = sfde.SFDE(0.6, 0.7, 2.0, 0.5, n, n, t)
    U0 = manufactured_initial(n, n, "10exp(-t)")
    F = manufactured_forcing(n, n, t, 0.6, 0.7, 2.0, 0.5, "10exp(-t)")
    r = mgrit.mgrit_modal(P, U0, F, m=m, max_levels=2, coarse="cn", rel_tol=1e-13, max_iter=40,
                          init_seed=1)
    fac = r.conv_factor_last5
    printed = tab["beta0.6_gamma0.7"][key]
    assert 0.4 * printed < fac < 2.5 * printed, fac
    bound = analysis.tub_bound(P.sigma(), t, m, "cn")
    assert fac <= bound * 1.05, (fac, bound)


def test_stiff_crank_nicolson_bound_exceeds_one():
    """For large dt*sigma the bound of Theorem 3.1 with the CN coarse propagator exceeds 1 (the
    iteration can grow), while the L-stable backward-Euler coarse propagator stays below it."""
    n = 31
    t = time_grid(128)
    P = sfde.SFDE(0.6, 0.9, 1.0, 0.5, n, n, t)
    assert analysis.tub_bound(P.sigma(), t, 8, "cn") > 1.0
    assert analysis.tub_bound(P.sigma(), t, 8, "be") < analysis.tub_bound(P.sigma(), t, 8, "cn")


def test_tub_bound_single_mode_by_hand():
    """Eq. (3.11) for one mode on a uniform grid, evaluated by hand in rationals.

    sigma = 1, dt = 1/2, m = 2, N_t = 8 (N_c = 4): lambda = (2 - 1/2)/(2 + 1/2) = 3/5,
    mu (CN, coarse step 1) = (2 - 1)/(2 + 1) = 1/3, so the bound is
    (3/5)^2 |(3/5)^2 - 1/3| (1 - (1/3)^3)/(1 - 1/3) = 9/25 * 2/75 * 13/9 = 26/1875.
    sigma = 10: lambda = (2 - 5)/(2 + 5) = -3/7 (lambda^dagger = 3/7), mu = (2 - 10)/(2 + 10) = -2/3
    (mu^ddagger = -2/3, mu^* = 2/3): (3/7)^2 |(3/7)^2 + 2/3| (1 - (2/3)^3)/(1/3) = 2375/7203.
    Both modes together: the larger, 2375/7203.  Backward-Euler coarse propagator, sigma = 1:
    mu = 1/(1 + 1) = 1/2: 9/25 |9/25 - 1/2| (1 - 1/8)/(1/2) = 9/25 * 7/50 * 7/4 = 441/5000."""
    from fractions import Fraction as Fr
    t = np.linspace(0.0, 4.0, 9)          # dt = 1/2
    assert analysis.tub_bound(np.array([1.0]), t, 2, "cn") == pytest.approx(float(Fr(26, 1875)), rel=1e-14)
    assert analysis.tub_bound(np.array([10.0]), t, 2, "cn") == pytest.approx(float(Fr(2375, 7203)), rel=1e-14)
    assert analysis.tub_bound(np.array([1.0, 10.0]), t, 2, "cn") == pytest.approx(float(Fr(2375, 7203)), rel=1e-14)
    assert analysis.tub_bound(np.array([1.0]), t, 2, "be") == pytest.approx(float(Fr(441, 5000)), rel=1e-14)


def test_space_time_residual_against_assembled_kronecker_rows():
    """rho_n = F_n + B_n U_{n-1} - S_n U_n evaluated with the assembled Kronecker matrices of
    Eq. (2.4) (row-major vec), on an arbitrary field; and zero (to rounding) on the sequential
    solution, which satisfies every row of Eq. (3.1)."""
    P, U0, F = _small(nt=6, grid="graded", nx=4, ny=3)
    rng = np.random.default_rng(3)
    U = rng.standard_normal((7, 3, 4))
    rho = mgrit.space_time_residual(P, U, F)
    Mk = np.kron(P.My, P.Mx)
    Kk = P.kx * np.kron(P.My, P.Ax) + P.ky * np.kron(P.Ay, P.Mx)
    for n in range(1, 7):
        tau = 0.5 * (P.t[n] - P.t[n - 1])
        want = F.dense(n).reshape(-1) + (Mk - tau * Kk) @ U[n - 1].reshape(-1) - (Mk + tau * Kk) @ U[n].reshape(-1)
        np.testing.assert_allclose(rho[n - 1].reshape(-1), want, rtol=0, atol=1e-14 * np.abs(want).max())
    seq = sfde.seq_timestep(P, U0, F, dense=True)
    assert np.abs(mgrit.space_time_residual(P, seq, F)).max() < 1e-14 * np.abs(seq).max()


def test_sform_residual_of_f_consistent_iterate_is_S_times_cpoint_residual():
    """After FCF (or F) relaxation every F-point satisfies its row of Eq. (3.1), so the space-time
    residual vanishes there and equals S_{km} r_k at the C-points, r_k = Phi_{km}(u_{km-1}) - u_{km}
    (S_n Phi_n(v) = B_n v + F_n): the identity the GPU's FP64 S-form stopping test uses."""
    P, U0, F = _small(nt=16, grid="graded", nx=5, ny=4)
    m = 4
    r = mgrit.mgrit(P, U0, F, m=m, max_levels=2, rel_tol=0.0, max_iter=1, init_seed=5, dense=True)
    u = r.U.copy()
    # one more FCF relaxation of the returned iterate, as the solver does before its test
    for sweep in ("F", "C", "F"):
        for n in range(1, 17):
            if (sweep == "F") == (n % m != 0):
                u[n] = P.step(u[n - 1], n, F.dense(n), dense=True)
    rho = mgrit.space_time_residual(P, u, F)
    scale = np.abs(rho).max()
    for n in range(1, 17):
        if n % m:
            assert np.abs(rho[n - 1]).max() < 1e-13 * scale, n
        else:
            rk = P.step(u[n - 1], n, F.dense(n), dense=True) - u[n]
            tau = 0.5 * (P.t[n] - P.t[n - 1])
            np.testing.assert_allclose(rho[n - 1], P.apply_S(rk, tau), rtol=0, atol=1e-13 * scale)


@pytest.mark.parametrize("stop", ["cpoint", "sform"])
def test_skip_first_down_keeps_the_fixed_point(stop):
    """With the first down-cycle skipped (Sec. 3.2), the iteration still converges to sequential
    stepping, and its first iteration runs only the level-0 C-point residual steps, the coarse
    levels' residual steps and the coarsest sweep on the way down, plus the up-cycle's F-relaxations:
    no relaxation on the down-cycle."""
    P, U0, F = _small(nt=32, grid="graded")
    seq = sfde.seq_timestep(P, U0, F, dense=True)
    r = mgrit.mgrit(P, U0, F, m=2, max_levels=3, rel_tol=1e-12, max_iter=60, dense=True,
                    skip_first_down=True, stop=stop)
    assert r.converged
    assert np.abs(r.U - seq).max() <= 1e-10 * np.abs(seq).max()
    one = mgrit.mgrit(P, U0, F, m=2, max_levels=3, rel_tol=0.0, max_iter=1, skip_first_down=True, stop=stop)
    # levels 32 -> 16 -> 8: residual steps 16 (level 0) + 8 (level 1), coarsest 8 steps,
    # up-cycle F-relaxation of level 1 (8 steps); no F/C relaxation on levels 0 and 1 going down
    assert one.step_solves == 16 + 8 + 8 + 8
    full = mgrit.mgrit(P, U0, F, m=2, max_levels=3, rel_tol=0.0, max_iter=1, stop=stop)
    # FCF on level 0 (16 + 16 + 16) and level 1 (8 + 8 + 8) on the way down in addition
    assert full.step_solves == one.step_solves + 48 + 24
