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
