"""The C-ABI library builds, loads without a GPU and exports every entry point of include/sfde.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions(headers=("sfde.h",)):
    src = "".join(open(os.path.join(ROOT, "include", h)).read() for h in headers)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:sfde_status|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def _library():
    import paper_1805_06688_gb300 as sfde
    if not os.path.exists(sfde.library_path):
        pytest.importorskip("shutil")
        from paper_1805_06688_gb300.build import build
        build()
    return sfde


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("sfde_setup", "mgrit_solve", "seq_timestep", "sfde_destroy", "sfde_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    sfde = _library()
    lib = ctypes.CDLL(sfde.library_path)
    headers = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    missing = [n for n in _declared_functions(headers) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared_functions()) <= set(sfde.exported_symbols) | {"sfde_zz_placeholder"}


def test_argument_validation_needs_no_gpu():
    """Invalid arguments are rejected before any CUDA call."""
    import numpy as np
    sfde = _library()
    L = sfde.lib()
    t = np.linspace(0, 1, 5)
    bad_t = np.array([0.0, 0.5, 0.4, 1.0, 1.1])
    ctx = ctypes.c_void_p()
    om = np.array([0.0, 1.0, 0.0, 1.0])
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cases = [
        (0.5, 0.8, 1.0, 1.0, 5, 5, t),      # beta not in (1/2, 1]
        (0.7, 1.2, 1.0, 1.0, 5, 5, t),      # gamma too large
        (0.7, 0.8, -1.0, 1.0, 5, 5, t),     # K_x <= 0
        (0.7, 0.8, 1.0, 1.0, 0, 5, t),      # N_x < 1
        (0.7, 0.8, 1.0, 1.0, 5, 5, bad_t),  # non-increasing grid
    ]
    for b, g, kx, ky, nx, ny, tt in cases:
        st = L.sfde_setup(b, g, kx, ky, dp(om), nx, ny, dp(tt), len(tt) - 1, None, ctypes.byref(ctx))
        assert st == sfde.SFDE_EINVAL
    assert L.mgrit_solve(None, None, None, None, None) == sfde.SFDE_EINVAL
    assert sfde.sfde_strerror(sfde.SFDE_ENOCONV) == "no convergence"


def test_batch_solve_argument_validation_needs_no_gpu():
    """sfde_batch_solve rejects an empty batch and NULL contexts before any CUDA call."""
    import ctypes as C
    sfde = _library()
    L = sfde.lib()
    assert L.sfde_batch_solve(0, None, None, None, None, None) == sfde.SFDE_EINVAL
    arr = (C.c_void_p * 2)(None, None)
    assert L.sfde_batch_solve(2, arr, None, None, None, None) == sfde.SFDE_EINVAL


def _inner_levels(L, nt, m, max_levels=32, min_coarse=2):
    sizes = (ctypes.c_int * 16)()
    count = ctypes.c_int()
    st = L.sfde_debug_inner_levels(nt, m, max_levels, min_coarse, sizes, 16, ctypes.byref(count))
    return st, list(sizes[:min(count.value, 16)])


def test_inner_hierarchy_rule_needs_no_gpu():
    """The mixed solver's inner hierarchy (host rule): coarsen by m while it divides and the coarse
    level keeps min_coarse points; stop at a coarse level whose direct sweep (N steps) is no longer
    than relaxing it (3m - 1 steps) plus the sweep below."""
    sfde = _library()
    L = sfde.lib()
    L.sfde_debug_inner_levels.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                                ctypes.POINTER(ctypes.c_int)]
    # the benchmark: 1024 -> 128 -> 16 (16 <= 23 + 2 stops there, 128 > 23 + 16 does not)
    assert _inner_levels(L, 1024, 8) == (0, [1024, 128, 16])
    assert _inner_levels(L, 4096, 16) == (0, [4096, 256, 16])
    assert _inner_levels(L, 64, 4, max_levels=3) == (0, [64, 16, 4])
    assert _inner_levels(L, 96, 4, max_levels=8) == (0, [96, 24, 6])      # 6 is not divisible by 4
    assert _inner_levels(L, 1024, 8, max_levels=2) == (0, [1024, 128])
    assert _inner_levels(L, 1024, 8, max_levels=1) == (0, [1024])
    assert _inner_levels(L, 100, 8) == (0, [100])                          # m does not divide N_t
    assert _inner_levels(L, 64, 8, min_coarse=16) == (0, [64])             # 8 < min_coarse
    assert _inner_levels(L, 64, 4, max_levels=8) == (0, [64, 16, 4])       # 16 > 11 + 4: relaxed
    for bad in ((0, 8, 32, 2), (64, 1, 32, 2), (64, 4, 0, 2), (64, 4, 8, 0)):
        assert _inner_levels(L, *bad)[0] == sfde.SFDE_EINVAL


def test_residual_digits_rule_needs_no_gpu():
    """Digits per operand of the tensor-core residual: the fewest nd in 4..7 whose products are
    accurate to 2^{9-8nd} <= 1e-5 prev / res0."""
    sfde = _library()
    L = sfde.lib()
    L.sfde_debug_residual_digits.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]

    def nd(prev, res0):
        v = ctypes.c_int()
        assert L.sfde_debug_residual_digits(prev, res0, ctypes.byref(v)) == 0
        return v.value

    assert nd(0.0, 1.0) == 4 and nd(1.0, 0.0) == 4 and nd(float("nan"), 1.0) == 4
    assert nd(1.0, 1.0) == 4          # need 1e-5: 2^-23 = 1.2e-7 suffices
    assert nd(2e-2, 1.0) == 4         # need 2e-7: 2^-23 = 1.2e-7 suffices
    assert nd(1e-2, 1.0) == 5         # need 1e-7: 2^-23 just too coarse
    assert nd(1e-3, 1.0) == 5         # need 1e-8: 2^-23 too coarse, 2^-31 = 4.7e-10
    assert nd(1e-6, 1.0) == 6         # need 1e-11: 2^-39 = 1.8e-12
    assert nd(1e-9, 1.0) == 7         # need 1e-14: 2^-47 = 7.1e-15
    assert nd(1e-20, 1.0) == 7        # capped
    assert nd(3e-4, 3.0) == nd(1e-4, 1.0)


@pytest.mark.parametrize("grid,m,coarse", [("uniform", 8, "cn"), ("uniform", 4, "be"), ("graded", 4, "cn"),
                                           ("graded", 8, "be")])
def test_theorem31_bound_matches_oracle(grid, m, coarse):
    """The Theorem 3.1 bound (3.11) that picks the coarse propagator under COARSE_AUTO (host code of
    the library, extremes over the steps) equals the oracle's evaluation over every step size."""
    import numpy as np
    from oracle import analysis
    from oracle import sfde as osfde
    from sfde_workloads import time_grid
    sfde = _library()
    L = sfde.lib()
    dp = ctypes.POINTER(ctypes.c_double)
    L.sfde_debug_tub_bound.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
    nt = 64
    t = time_grid(nt, 1.0, grid)
    P = osfde.SFDE(0.7, 0.85, 1.3, 0.6, 23, 17, t)
    lx, _, ly, _ = P.eig()
    ref = analysis.tub_bound(P.sigma(), t, m, coarse)
    out = ctypes.c_double()
    c = {"cn": sfde.COARSE_CN, "be": sfde.COARSE_BE}[coarse]
    st = L.sfde_debug_tub_bound(np.ascontiguousarray(lx).ctypes.data_as(dp), len(lx),
                                np.ascontiguousarray(ly).ctypes.data_as(dp), len(ly), 1.3, 0.6,
                                np.ascontiguousarray(t).ctypes.data_as(dp), nt, m, c, ctypes.byref(out))
    assert st == 0
    assert abs(out.value - ref) <= 1e-12 * max(1.0, abs(ref)), (out.value, ref)
    st = L.sfde_debug_tub_bound(np.ascontiguousarray(lx).ctypes.data_as(dp), len(lx),
                                np.ascontiguousarray(ly).ctypes.data_as(dp), len(ly), 1.3, 0.6,
                                np.ascontiguousarray(t).ctypes.data_as(dp), nt, m, 7, ctypes.byref(out))
    assert st == sfde.SFDE_EINVAL


def _tuning_lib():
    sfde = _library()
    L = sfde.lib()
    tp = ctypes.POINTER(sfde.SfdeTuning)
    L.sfde_debug_tune_pick.argtypes = [tp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.sfde_debug_tune_cache.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int, tp,
                                        ctypes.POINTER(ctypes.c_int)]
    return sfde, L


def test_autotune_pick_needs_no_gpu():
    """The autotuner keeps the fastest measured choice: smallest positive finite time, the first on
    ties; unmeasured (0), failed (inf, nan) and negative entries never win."""
    sfde, L = _tuning_lib()
    T = sfde.SfdeTuning

    def pick(times):
        arr = (T * max(1, len(times)))(*[T(1, 1, 0, v) for v in times])
        best = ctypes.c_int()
        assert L.sfde_debug_tune_pick(arr, len(times), ctypes.byref(best)) == 0
        return best.value

    assert pick([]) == -1
    assert pick([0.0, 0.0]) == -1
    assert pick([5.0, 3.0, 4.0]) == 1
    assert pick([3.0, 5.0, 3.0]) == 0
    assert pick([float("inf"), float("nan"), -1.0, 0.0, 7.5]) == 4
    assert L.sfde_debug_tune_pick(None, 2, ctypes.byref(ctypes.c_int())) == sfde.SFDE_EINVAL


def test_autotune_cache_file_needs_no_gpu(tmp_path):
    """The tuning cache: one text line per measurement, the last valid line for a key counts,
    other keys and malformed or out-of-range lines are ignored, a missing file is a miss."""
    sfde, L = _tuning_lib()
    T = sfde.SfdeTuning
    path = str(tmp_path / "tune.txt").encode()
    found = ctypes.c_int(7)
    t = T()
    assert L.sfde_debug_tune_cache(path, b"P256x256_nt1024", 0, ctypes.byref(t), ctypes.byref(found)) == 0
    assert found.value == 0
    for key, v in ((b"P256x256_nt1024", T(1, 1, 0, 55.4)), (b"P512x512_nt2048", T(1, 3, 5, 900.0)),
                   (b"P256x256_nt1024", T(3, 3, 0, 52.4))):
        assert L.sfde_debug_tune_cache(path, key, 1, ctypes.byref(v), None) == 0
    with open(path, "a") as f:
        f.write("P256x256_nt1024 9 1 0 1.0\n")        # fused_pair out of range: skipped
        f.write("P256x256_nt1024 1 1\n")              # malformed: skipped
        f.write("\n")
    assert L.sfde_debug_tune_cache(path, b"P256x256_nt1024", 0, ctypes.byref(t), ctypes.byref(found)) == 0
    assert found.value == 1 and (t.fused_pair, t.modal_chains, t.inner_cycles) == (3, 3, 0)
    assert abs(t.ms - 52.4) < 1e-9
    assert L.sfde_debug_tune_cache(path, b"P512x512_nt2048", 0, ctypes.byref(t), ctypes.byref(found)) == 0
    assert found.value == 1 and (t.fused_pair, t.modal_chains, t.inner_cycles) == (1, 3, 5)
    assert L.sfde_debug_tune_cache(path, b"P128x128_nt64", 0, ctypes.byref(t), ctypes.byref(found)) == 0
    assert found.value == 0
    bad = T(1, 5, 0, 1.0)
    assert L.sfde_debug_tune_cache(path, b"k", 1, ctypes.byref(bad), None) == sfde.SFDE_EINVAL
    assert L.sfde_debug_tune_cache(path, b"two words", 0, ctypes.byref(t), ctypes.byref(found)) == sfde.SFDE_EINVAL
    assert L.sfde_debug_tune_cache(path, b"", 0, ctypes.byref(t), ctypes.byref(found)) == sfde.SFDE_EINVAL


def test_set_tuning_and_autotune_validate_arguments_without_gpu():
    sfde, L = _tuning_lib()
    t = sfde.SfdeTuning(1, 1, 0, 0.0)
    assert L.sfde_set_tuning(None, ctypes.byref(t)) == sfde.SFDE_EINVAL
    assert L.sfde_autotune(None, None, None, None) == sfde.SFDE_EINVAL
    L.sfde_get_tuning.argtypes = [ctypes.c_void_p, ctypes.POINTER(sfde.SfdeTuning)]
    assert L.sfde_get_tuning(None, ctypes.byref(t)) == sfde.SFDE_EINVAL


def test_step_buffer_checks_refuse_bad_input_without_gpu():
    """The binding refuses, before any call into C, step buffers that are too short, overlap, or (for
    the no-allocation entry point) are not CUDA tensors: the C side cannot know buffer sizes, and a
    short buffer would be read or written past its end by the pad and unpad kernels."""
    import numpy as np
    from paper_1805_06688_gb300 import _binding as B
    key = 0x7F00DEAD0000
    B._CTX_DIMS[key] = (5, 4, 8)            # nx, ny, nt of a stand-in context (no GPU needed)
    try:
        ok = np.zeros((2, 4, 5))
        short = np.zeros((1, 4, 5))
        with pytest.raises(ValueError, match="needs"):
            B.sfde_step_batch(key, 1, 1, 2, short, ok)
        with pytest.raises(ValueError, match="needs"):
            B.sfde_step_batch(key, 1, 1, 2, ok, short)
        with pytest.raises(ValueError, match="overlap"):
            B.sfde_step_batch(key, 1, 1, 1, ok, ok)
        with pytest.raises(ValueError, match="overlap"):
            flat = np.zeros(3 * 20)
            B.sfde_step_batch(key, 1, 1, 2, flat[:40], flat[20:])
        with pytest.raises(ValueError, match="batch"):
            B.sfde_step_batch(key, 1, 1, 0, ok, ok.copy())
        with pytest.raises(ValueError, match="CUDA"):
            B.sfde_step_batch_noalloc(key, 1, 1, 1, ok, ok.copy())
        with pytest.raises(ValueError, match="float64"):
            B.sfde_step_batch(key, 1, 1, 1, ok.astype(np.float32), ok.copy())
        with pytest.raises(ValueError, match="unknown"):
            B.sfde_step_batch(key + 8, 1, 1, 1, ok, ok.copy())
    finally:
        B._CTX_DIMS.pop(key, None)


@pytest.mark.parametrize("rho", [0.55, 0.75, 0.95, 1.0])
def test_p1_entries_match_the_printed_formulas_without_gpu(rho):
    """The library's evaluation of the printed A_1 / A_2 entries of Sec. 2 (direct sums for offsets
    below 16, a binomial series of the differences above) against the oracle's 40-digit evaluation
    of the printed formulas, up to offset 1100."""
    import numpy as np
    from oracle import p1
    sfde = _library()
    L = sfde.lib()
    dp = ctypes.POINTER(ctypes.c_double)
    L.sfde_debug_p1_entries.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp]
    n = 1100
    a1, up, lo = np.zeros(n), np.zeros(n), np.zeros(n)
    assert L.sfde_debug_p1_entries(n, rho, a1.ctypes.data_as(dp), up.ctypes.data_as(dp), lo.ctypes.data_as(dp)) == 0
    idx = sorted(set(list(range(0, 40)) + list(range(40, n, 37)) + [n - 1]))
    scale = abs(p1.a1(0, rho))
    for l in idx:
        ref = (p1.a1(l, rho), p1.a2_upper(l, rho), p1.a2_lower(l, rho) if l else 0.0)
        for got, want in zip((a1[l], up[l], lo[l]), ref):
            assert abs(got - want) <= 3e-12 * abs(want) + 1e-15 * scale, (l, got, want)
    assert L.sfde_debug_p1_entries(0, rho, a1.ctypes.data_as(dp), up.ctypes.data_as(dp), lo.ctypes.data_as(dp)) == \
        sfde.SFDE_EINVAL


def test_p1_operator_options_are_validated_without_gpu():
    """operator_kind outside {0, 1} is invalid; the P1 operator runs in FP64 only."""
    import numpy as np
    sfde = _library()
    L = sfde.lib()
    t = np.linspace(0, 1, 5)
    om = np.array([0.0, 1.0, 0.0, 1.0])
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ctx = ctypes.c_void_p()
    for prec, op, want in ((0, 2, sfde.SFDE_EINVAL), (0, -1, sfde.SFDE_EINVAL), (1, 1, sfde.SFDE_EUNSUPPORTED),
                           (3, 1, sfde.SFDE_EUNSUPPORTED)):
        o = sfde.SfdeOpts(prec, None, op)
        st = L.sfde_setup(0.7, 0.8, 1.0, 1.0, dp(om), 5, 5, dp(t), 4, ctypes.byref(o), ctypes.byref(ctx))
        assert st == want, (prec, op, st)
