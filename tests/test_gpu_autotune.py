"""The autotuner end to end on a small mixed-precision problem: the winner is a valid candidate and is
what the context applies afterwards; a second call with the same cache file finds the choice there and
runs no trial solve (no kernel launch); when no candidate converges the previous choice stays; a solve
after tuning (inner graphs captured again for the new choice) matches the oracle's exact sequential
solution of Eq. (2.4)."""
import numpy as np
import pytest

from oracle import sfde as osfde
from sfde_workloads import gaussian_bump_forcing, sine_mode_amplitudes, sine_mode_nodal, time_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_06688_gb300 as sfde  # noqa: E402

NX = NY = 63
NT = 32
OPTS = dict(m=4, max_levels=3, coarse=sfde.COARSE_BE, rel_tol=1e-11, max_iter=60, stop_kind=sfde.STOP_SFORM)


def _problem(prec):
    t = time_grid(NT, 1.0, "uniform")
    F, _ = gaussian_bump_forcing(3, NX, NY, t)
    psi = sine_mode_nodal(sine_mode_amplitudes(4), NX, NY)
    P = sfde.Problem(0.6, 0.9, 1.0, 0.5, NX, NY, t, precision=prec)
    P.set_initial(psi)
    P.set_forcing(F)
    return P, t, psi, F


def _fields(t):
    return (t.fused_pair, t.modal_chains, t.inner_cycles)


@pytest.mark.parametrize("prec", [sfde.PREC_MIXED_BF16, sfde.PREC_MIXED_TF32])
def test_autotune_applies_caches_and_keeps_the_fixed_point(prec, tmp_path):
    P, t, psi, F = _problem(prec)
    cache = tmp_path / "tune.txt"
    win = P.autotune(cache_path=str(cache), **OPTS)
    # a candidate of the fixed grid: eigenbasis on the coarse levels or every level, 3/5 or default
    # V-cycles, the whole inner solve in the eigenbasis (FP32 storage) with 3/5/8 or default V-cycles,
    # or a forced CTA-pair form of the fused step
    full = {(4, 0), (4, 3), (4, 5), (4, 8)} if prec != sfde.PREC_MIXED_BF16 else set()
    assert (win.modal_chains, win.inner_cycles) in {(1, 0), (1, 3), (1, 5), (2, 0), (2, 3), (2, 5)} | full or \
        (win.fused_pair in (2, 3) and win.modal_chains == 1 and win.inner_cycles == 0)
    assert win.ms > 0.0 and np.isfinite(win.ms)
    assert _fields(P.tuning()) == _fields(win)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].split()[1:4] == [str(v) for v in _fields(win)]

    # the cache hit: another choice set by hand, then the stored one comes back without a trial solve
    P.set_tuning(fused_pair=0, modal_chains=0, inner_cycles=7)
    assert _fields(P.tuning()) == (0, 0, 7)
    P.profile_enable(True)
    before = P.profile_read().kernel_launches
    again = P.autotune(cache_path=str(cache), **OPTS)
    assert P.profile_read().kernel_launches == before
    P.profile_enable(False)
    assert _fields(again) == _fields(win) and _fields(P.tuning()) == _fields(win)
    assert len(cache.read_text().splitlines()) == 1

    # a solve with the tuned choice matches the exact sequential solution
    U = np.zeros((NT + 1, NY, NX))
    _, st = P.mgrit(U=U, **OPTS)
    assert st.converged
    ref = osfde.seq_timestep(osfde.SFDE(0.6, 0.9, 1.0, 0.5, NX, NY, t), psi, F)
    assert float(np.abs(U - ref).max() / np.abs(ref).max()) < 1e-8


def test_autotune_without_a_converging_candidate_keeps_the_previous_choice(tmp_path):
    P, *_ = _problem(sfde.PREC_MIXED_BF16)
    P.set_tuning(fused_pair=1, modal_chains=0, inner_cycles=2)
    cache = tmp_path / "tune.txt"
    opts = dict(OPTS, rel_tol=1e-12, max_iter=1)   # one refinement step cannot reach 1e-12
    with pytest.raises(sfde.SfdeError) as e:
        P.autotune(cache_path=str(cache), **opts)
    assert e.value.status == sfde.SFDE_ENOCONV
    assert _fields(P.tuning()) == (1, 0, 2)
    assert not cache.exists() or cache.read_text() == ""


def test_fp64_context_has_nothing_to_tune(tmp_path):
    P, *_ = _problem(sfde.PREC_FP64)
    cur = _fields(P.tuning())
    P.profile_enable(True)
    before = P.profile_read().kernel_launches
    got = P.autotune(cache_path=str(tmp_path / "t.txt"), **OPTS)
    assert P.profile_read().kernel_launches == before
    assert _fields(got) == cur
    assert not (tmp_path / "t.txt").exists()
