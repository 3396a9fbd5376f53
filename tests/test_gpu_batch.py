"""The batched form (sfde_batch_solve): independent instances of different sizes, grids and
precisions solved concurrently give exactly the results of separate solves, and each matches the
oracle's exact sequential solution at t_N to 1e-8 (mixed forms) or 1e-10 (FP64) of the solution's
size over the space-time grid (max of |psi_0| and |u(T)|): the stopping test bounds the space-time
residual, and u(T) itself may have decayed by orders of magnitude."""
import numpy as np
import pytest

from oracle import sfde as osfde
from sfde_workloads import gaussian_bump_forcing, sine_mode_amplitudes, sine_mode_nodal, time_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_06688_gb300 as sfde  # noqa: E402

# (beta, gamma, kx, ky, nx, ny, nt, grid, precision, forcing seed or None)
INSTANCES = [
    (0.6, 0.9, 1.0, 0.5, 63, 63, 128, "uniform", sfde.PREC_MIXED_AUTO, None),
    (0.75, 0.8, 0.3, 1.7, 127, 100, 64, "graded", sfde.PREC_MIXED_BF16, 3),
    (0.55, 0.95, 1.0, 0.1, 255, 255, 256, "uniform", sfde.PREC_MIXED_AUTO, None),
    (0.9, 0.6, 2.0, 0.2, 200, 150, 96, "uniform", sfde.PREC_MIXED_TF32, 5),
    (0.7, 0.7, 1.0, 1.0, 40, 31, 64, "graded", sfde.PREC_FP64, None),
    (0.65, 0.85, 1.5, 0.7, 300, 260, 64, "uniform", sfde.PREC_MIXED_BF16, None),
]
KW = dict(m=4, max_levels=8, coarse=sfde.COARSE_AUTO, rel_tol=1e-10, max_iter=100)


def make(inst):
    b, g, kx, ky, nx, ny, nt, grid, prec, fseed = inst
    t = time_grid(nt, 1.0, grid)
    psi = sine_mode_nodal(sine_mode_amplitudes(nx + ny), nx, ny)
    F = gaussian_bump_forcing(fseed, nx, ny, t)[0] if fseed is not None else None
    P = sfde.Problem(b, g, kx, ky, nx, ny, t, precision=prec)
    P.set_initial(psi)
    P.set_forcing(F)
    return P, psi, F, t


def test_batch_equals_separate_solves_and_oracle():
    built = [make(i) for i in INSTANCES]
    probs = [p for p, *_ in built]
    UT = [np.zeros((i[5], i[4])) for i in INSTANCES]
    st, status, stats = sfde.batch_solve(probs, U_T=UT, **KW)
    assert st == sfde.SFDE_OK and all(s == 0 for s in status), status
    assert all(s.converged for s in stats)
    for inst, (P, psi, F, t), ut in zip(INSTANCES, built, UT):
        Q = make(inst)[0]
        ref = np.zeros_like(ut)
        Q.mgrit(U_T=ref, **KW)
        assert np.array_equal(ut, ref)
        b, g, kx, ky, nx, ny, nt = inst[:7]
        O = osfde.SFDE(b, g, kx, ky, nx, ny, t)
        exact = osfde.spectral_sequential(O, psi, F, keep=[nt])[nt]
        tol = 1e-10 if inst[8] == sfde.PREC_FP64 else 1e-8
        scale = max(np.abs(psi).max(), np.abs(exact).max())
        assert np.abs(ut - exact).max() <= tol * scale, inst


def test_batch_rejects_repeated_contexts():
    P = make(INSTANCES[0])[0]
    with pytest.raises(sfde.SfdeError):
        sfde.batch_solve([P, P], **KW)


def test_batch64_uneven_instances_against_oracle():
    """The batched form on all 64 instances of the uneven batch (N in {63, 127, 255, 511}, N_t in
    {256, 512, 1024, 4096}, random orders and diffusivities, sine-mode psi_0, f = 0), operands chosen
    per instance, stopped on the FP64 space-time residual at 1e-8: every instance converges and its
    u(T) matches the oracle's exact sequential solution to 1e-8 of the solution's size."""
    from concurrent.futures import ThreadPoolExecutor
    from sfde_workloads.generate import batch_workloads
    ws = batch_workloads(0, 64)
    probs, UT = [], []
    for w in ws:
        P = sfde.Problem(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, w.t(), w.omega, precision=sfde.PREC_MIXED_AUTO)
        P.set_initial(w.initial())
        probs.append(P)
        UT.append(np.zeros((w.ny, w.nx)))
    st, status, stats = sfde.batch_solve(probs, U_T=UT, m=8, max_levels=32, coarse=sfde.COARSE_AUTO, rel_tol=1e-8,
                                         max_iter=200, stop_kind=sfde.STOP_SFORM)
    assert st == sfde.SFDE_OK and all(s == 0 for s in status), status
    assert all(s.converged for s in stats)

    def check(k):
        w = ws[k]
        O = osfde.SFDE(w.beta, w.gamma, w.kx, w.ky, w.nx, w.ny, w.t(), w.omega)
        psi = w.initial()
        exact = osfde.spectral_sequential(O, psi, None, keep=[w.nt])[w.nt]
        scale = max(np.abs(psi).max(), np.abs(exact).max())
        return float(np.abs(UT[k] - exact).max() / scale)

    with ThreadPoolExecutor(max_workers=8) as ex:
        errs = list(ex.map(check, range(len(ws))))
    worst = int(np.argmax(errs))
    assert max(errs) <= 1e-8, (ws[worst].name, errs[worst])
