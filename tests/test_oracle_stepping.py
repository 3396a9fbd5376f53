"""Pins of the oracle's step solve and sequential stepping (Eq. (2.4), Eqs. (3.5)-(3.7))."""
import json
import math
import os

import numpy as np
import pytest

from oracle import sfde
from sfde_workloads import (manufactured_exact, manufactured_forcing, manufactured_initial,
                            gaussian_bump_forcing, time_grid, sine_mode_amplitudes, sine_mode_nodal)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def _prob(nx=5, ny=7, nt=8, grid="uniform", beta=0.6, gamma=0.9, kx=1.3, ky=0.4, omega=(0, 1, 0, 2)):
    return sfde.SFDE(beta, gamma, kx, ky, nx, ny, time_grid(nt, 1.0, grid), omega)


def test_operator_equals_assembled_kronecker():
    P = _prob()
    U = np.random.default_rng(1).standard_normal((P.ny, P.nx))
    for tau in (0.0, 0.013, 2.5):
        np.testing.assert_allclose(P.apply_S(U, tau).reshape(-1), P.kron_S(tau) @ U.reshape(-1),
                                   rtol=1e-13, atol=1e-13)
    # the assembled operator is symmetric positive definite (Lemma 3.2)
    S = P.kron_S(0.3)
    assert np.allclose(S, S.T)
    np.linalg.cholesky(S)


def test_fdm_step_equals_dense_solve():
    P = _prob(grid="graded")
    rng = np.random.default_rng(2)
    U = rng.standard_normal((P.ny, P.nx))
    F = rng.standard_normal((P.ny, P.nx))
    for n in (1, 4, 8):
        a = P.step(U, n, F, dense=True)
        b = P.step(U, n, F, dense=False)
        assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
    for dt in (1e-3, 0.7):
        for scheme in ("cn", "be"):
            a = P.propagate(U, dt, scheme, dense=True)
            b = P.propagate(U, dt, scheme)
            assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def test_generalised_eigenpairs():
    P = _prob(nx=11, ny=9)
    lx, Vx, ly, Vy = P.eig()
    np.testing.assert_allclose(Vx.T @ P.Mx @ Vx, np.eye(11), atol=1e-12)
    np.testing.assert_allclose(Vx.T @ P.Ax @ Vx, np.diag(lx), atol=1e-10 * lx.max())
    assert lx.min() > 0 and ly.min() > 0  # Lemma 3.2: sigma real and positive


def test_rho_one_eigenvalues_closed_form():
    """For rho = 1, (A, M) = ((1/h) tridiag(-1,2,-1), (h/6) tridiag(1,4,1)) has the sine
    eigenvalues lambda_k = (6/h^2)(1 - cos k pi h)/(2 + cos k pi h)."""
    n = 15
    h = 1.0 / (n + 1)
    P = sfde.SFDE(1.0, 1.0, 1.0, 1.0, n, n, time_grid(2))
    lx = P.eig()[0]
    k = np.arange(1, n + 1)
    ref = 6.0 / h ** 2 * (1 - np.cos(k * np.pi * h)) / (2 + np.cos(k * np.pi * h))
    np.testing.assert_allclose(np.sort(lx), np.sort(ref), rtol=1e-12)


def test_propagator_eigenvalues_eq_3_7():
    """Psi x_w = lambda_w x_w with lambda_w = (2 - dt sigma_w)/(2 + dt sigma_w), |lambda| < 1."""
    P = _prob(nx=6, ny=5)
    lx, Vx, ly, Vy = P.eig()
    dt = 0.37
    for (j, i) in [(0, 0), (2, 3), (4, 5)]:
        X = np.outer(Vy[:, j], Vx[:, i])
        s = P.kx * lx[i] + P.ky * ly[j]
        lam = (2 - dt * s) / (2 + dt * s)
        assert abs(lam) < 1
        np.testing.assert_allclose(P.propagate(X, dt, "cn", dense=True), lam * X, atol=1e-12)


def test_spectral_recurrence_equals_stepping():
    P = _prob(nx=6, ny=8, nt=12, grid="graded", omega=(0, 1, 0, 1))
    U0 = sine_mode_nodal(sine_mode_amplitudes(3), 6, 8)
    F, _ = gaussian_bump_forcing(4, 6, 8, P.t)
    seq = sfde.seq_timestep(P, U0, F, dense=True)
    sp = sfde.spectral_sequential(P, U0, F)
    for n in range(P.nt + 1):
        assert np.abs(sp[n] - seq[n]).max() <= 1e-13 * np.abs(seq).max()


@pytest.mark.parametrize("scheme", ["cn", "be"])
def test_frelaxation_in_the_eigenbasis(scheme):
    """The identity the modal sweeps rest on: with W = M V (so W^T V = I, V^T M V = I), the chain
    u_j = Psi_j(u_{j-1}) + g_j of an F-relaxation (Algorithm 1, propagators (3.2)/(3.4)) is, for
    v = W_y^T u W_x, the per-mode recurrence v_j = lambda_j o v_{j-1} + W_y^T g_j W_x with the
    eigenvalues lambda of Eq. (3.7) -- checked against dense solves of the assembled Kronecker
    system on a graded grid, so a transposed W, a missing mass factor or the wrong eigenvalue
    (CN against BE) fails."""
    P = _prob(nx=6, ny=5, nt=7, grid="graded")
    rng = np.random.default_rng(11 if scheme == "cn" else 12)
    u = rng.standard_normal((5, 6))
    g = rng.standard_normal((P.nt, 5, 6))
    lx, Vx, ly, Vy = P.eig()
    Wx, Wy = P.Mx @ Vx, P.My @ Vy
    assert np.abs(Wx.T @ Vx - np.eye(6)).max() < 1e-12 and np.abs(Wy.T @ Vy - np.eye(5)).max() < 1e-12
    sig = P.sigma()
    v = Wy.T @ u @ Wx
    for j in range(1, P.nt + 1):
        dt = P.t[j] - P.t[j - 1]
        u = P.propagate(u, dt, scheme, dense=True) + g[j - 1]
        v = sfde.modal_lambda(sig, dt, scheme) * v + Wy.T @ g[j - 1] @ Wx
        assert np.abs(Vy @ v @ Vx.T - u).max() <= 1e-12 * np.abs(u).max(), j


def _example41_errors(beta, gamma, kx, ky, Ms, grid="uniform", eps=None):
    errs = []
    for M in Ms:
        n = M - 1
        t = time_grid(M, 1.0, grid, eps=eps)
        P = sfde.SFDE(beta, gamma, kx, ky, n, n, t)
        U0 = manufactured_initial(n, n, "10exp(-t)")
        F = manufactured_forcing(n, n, t, beta, gamma, kx, ky, "10exp(-t)")
        UT = sfde.seq_timestep(P, U0, F, keep_all=False)
        errs.append(sfde.l2_error_bilinear(UT, lambda X, Y: manufactured_exact(X, Y, 1.0, "10exp(-t)")))
    return np.array(errs)


@pytest.mark.parametrize("pair", ["beta0.6_gamma0.7", "beta0.95_gamma0.65", "beta0.8_gamma0.8"])
def test_saturation_error_order_example_4_1(pair):
    """Example 4.1, tau = h (Table 1 setting): O(h^2 + tau^2) error, rates near 2, and errors of
    the printed magnitude (the printed values are for P1 triangles; this operator is the
    tensor-product one, which differs from them by up to ~40% at these sizes)."""
    tab = json.load(open(GOLDEN))["table1"]
    b, g = (float(v) for v in pair.replace("beta", "").split("_gamma"))
    errs = _example41_errors(b, g, 2.0, 0.5, tab["M"])
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates > 1.75) and np.all(rates < 2.3), rates
    ratio = errs / np.array(tab[pair])
    assert np.all(ratio > 0.5) and np.all(ratio < 1.6), ratio


@pytest.mark.parametrize("pair", ["beta0.6_gamma0.7", "beta0.95_gamma0.65", "beta0.8_gamma0.8"])
def test_saturation_error_order_piecewise_uniform_grid(pair):
    """Example 4.1 on the piecewise uniform partition of Sec. 4.1 (Table 3 setting: N = 1/h,
    eps = 2^-6, K_x = 3.0, K_y = 7.5): the O(h^2 + tau^2) order carries over to the nonuniform
    steps, and the errors are of the printed magnitude (printed for P1 triangles; this is the
    tensor-product operator)."""
    tab = json.load(open(GOLDEN))["table3"]
    b, g = (float(v) for v in pair.replace("beta", "").split("_gamma"))
    errs = _example41_errors(b, g, 3.0, 7.5, tab["M"], "shishkin", tab["eps"])
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates > 1.75) and np.all(rates < 2.3), rates
    ratio = errs / np.array(tab[pair])
    assert np.all(ratio > 0.5) and np.all(ratio < 1.6), ratio


def test_moving_bump_load_reduces_to_the_separable_bump():
    """The dense load of a bump at rest (speed 0) is the separable Gaussian bump's space factors
    times the step length (the time integral of 1): pins the space-time quadrature of the dense load."""
    from sfde_workloads import moving_bump_dense_forcing
    from sfde_workloads.generate import _hat_load_gauss, interior_nodes
    t = time_grid(12, 1.0, "graded")
    D, (x0, y0, s, v) = moving_bump_dense_forcing(4, 9, 7, t, speed=0.0)
    assert v == 0.0
    bx = _hat_load_gauss(lambda z: np.exp(-(z - x0) ** 2 / (2 * s * s)), interior_nodes(9, 0.0, 1.0), 0.1)
    by = _hat_load_gauss(lambda z: np.exp(-(z - y0) ** 2 / (2 * s * s)), interior_nodes(7, 0.0, 1.0), 0.125)
    for n in range(1, 13):
        np.testing.assert_allclose(D.dense(n), (t[n] - t[n - 1]) * np.outer(by, bx), rtol=1e-14, atol=0)


def test_moving_bump_load_time_integral_is_exact_for_a_linear_path():
    """For a bump moving at speed v the x-factor integrates exp(-(x - x0 - v t)^2/(2 s^2)) over each
    step; with the 5-point Gauss rule in t this matches an adaptive quadrature of the same integrand
    at one node to 1e-12 (the integrand is smooth in t)."""
    from scipy.integrate import quad
    from sfde_workloads import moving_bump_dense_forcing
    t = time_grid(6)
    D, (x0, y0, s, v) = moving_bump_dense_forcing(8, 15, 3, t)
    assert v != 0.0
    h = 1.0 / 16
    i, j, n = 6, 1, 3                      # node x_7, y_2, step 3
    xi, yj = (i + 1) * h, (j + 1) * 0.25

    def hat(z, c, w):
        return max(0.0, 1.0 - abs(z - c) / w)

    def fx(tt):
        return quad(lambda z: np.exp(-(z - x0 - v * tt) ** 2 / (2 * s * s)) * hat(z, xi, h), xi - h, xi + h,
                    points=[xi], epsabs=1e-15, epsrel=1e-13)[0]

    gy = quad(lambda z: np.exp(-(z - y0) ** 2 / (2 * s * s)) * hat(z, yj, 0.25), yj - 0.25, yj + 0.25, points=[yj],
              epsabs=1e-15, epsrel=1e-13)[0]
    want = gy * quad(fx, t[n - 1], t[n], epsabs=1e-15, epsrel=1e-13)[0]
    assert abs(D.dense(n)[j, i] - want) <= 1e-9 * abs(want)


def test_spectral_sequential_with_dense_load_matches_dense_stepping():
    """The per-mode recurrence (Eq. (3.7)) with a dense, non-separable load equals sequential
    stepping by dense Kronecker solves, at every time point, streamed one slice at a time."""
    from oracle.sfde import spectral_sequential_iter
    from sfde_workloads import moving_bump_dense_forcing
    nx, ny, nt = 6, 5, 9
    t = time_grid(nt, 1.0, "graded")
    P = sfde.SFDE(0.65, 0.8, 1.2, 0.7, nx, ny, t)
    D, _ = moving_bump_dense_forcing(2, nx, ny, t)
    U0 = sine_mode_nodal(sine_mode_amplitudes(1), nx, ny)
    ref = sfde.seq_timestep(P, U0, D, dense=True)
    for n, U in spectral_sequential_iter(P, U0, D):
        assert np.abs(U - ref[n]).max() <= 1e-13 * np.abs(ref).max(), n
