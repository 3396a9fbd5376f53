"""FP64-accurate slice GEMM on BF16 tensor cores (error-free digit splitting) against an FP64 DGEMM.

Both results carry rounding errors of order K * 2^-53 * sum_k |x_k m_k|; the split product also
drops digit products below 2^-47 of 2^{e_r + e_n} K.  Tolerance: 1e-13 relative to
max_k|x_rk| * max_k|m_kn| * K per element (a plain BF16 or FP32 product would be off by ~1e-3/1e-7).
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_06688_gb300 as sfde  # noqa: E402


def run(X, Mat):
    batch, R, K = X.shape
    N = Mat.shape[1]
    out = torch.full((batch, N, R), float("nan"), dtype=torch.float64, device="cuda")
    err = ctypes.c_int(0)
    L = sfde.lib()
    L.sfde_debug_oz_gemm.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
    st = L.sfde_debug_oz_gemm(X.data_ptr(), batch, R, K, Mat.data_ptr(), N, out.data_ptr(), ctypes.byref(err))
    assert st == 0, (sfde.sfde_strerror(st), err.value)
    return out


@pytest.mark.parametrize("batch,R,K,N", [(3, 256, 256, 256), (5, 64, 64, 64), (7, 32, 32, 32), (2, 128, 256, 96),
                                         (1, 256, 128, 256)])
def test_ozaki_gemm_matches_fp64(batch, R, K, N):
    g = torch.Generator(device="cuda").manual_seed(batch * 131 + R + K + N)
    # rows and columns of very different magnitudes, as in the stiffness products
    X = torch.randn((batch, R, K), dtype=torch.float64, device="cuda", generator=g)
    X *= 10.0 ** (torch.rand((batch, R, 1), dtype=torch.float64, device="cuda", generator=g) * 8 - 4)
    Mat = torch.randn((K, N), dtype=torch.float64, device="cuda", generator=g)
    Mat *= 10.0 ** (torch.rand((1, N), dtype=torch.float64, device="cuda", generator=g) * 6 - 3)
    out = run(X, Mat)
    ref = torch.matmul(X, Mat).transpose(1, 2)
    scale = X.abs().amax(dim=2)[:, None, :] * Mat.abs().amax(dim=0)[None, :, None] * K
    rel = ((out - ref).abs() / scale).max().item()
    assert rel < 1e-13, rel


def test_ozaki_gemm_exact_on_small_integers():
    """Integer operands below 2^8 are one digit each: the product must be exact."""
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randint(-200, 200, (2, 128, 256), generator=g, device="cuda").double()
    Mat = torch.randint(-200, 200, (256, 64), generator=g, device="cuda").double()
    out = run(X, Mat)
    ref = torch.matmul(X, Mat).transpose(1, 2)
    assert torch.equal(out, ref)
