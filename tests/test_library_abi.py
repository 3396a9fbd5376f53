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
