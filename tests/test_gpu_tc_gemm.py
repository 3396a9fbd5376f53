"""The tcgen05/TMA slice GEMM against a float64 product of the same rounded operands.

BF16 operands multiply exactly into FP32, so the only difference is FP32 accumulation order:
error <= K * 2^-24 * sum|x||m|, tested as 1e-5 relative to the row/column magnitudes.
TF32 products drop the 13 low mantissa bits of each operand: tested at 2e-3 relative.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_06688_gb300 as sfde  # noqa: E402


def run(kind, X, s0, ds, batch, MatT):
    nslices, R, C = X.shape
    Cout = MatT.shape[0]
    out = torch.zeros((batch, Cout, R), dtype=X.dtype, device="cuda")
    err = ctypes.c_int(0)
    L = sfde.lib()
    L.sfde_debug_tc_gemm.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_float)]
    st = L.sfde_debug_tc_gemm(kind, X.data_ptr(), nslices, s0, ds, batch, R, C, MatT.data_ptr(), Cout,
                              out.data_ptr(), ctypes.byref(err), 0, None)
    assert st == 0, (sfde.sfde_strerror(st), err.value)
    return out


CASES = [
    # R, C, Cout, batch, s0, ds, nslices
    (256, 256, 256, 4, 0, 1, 4),
    (256, 256, 256, 16, 3, 8, 136),
    (64, 64, 64, 5, 1, 2, 12),
    (32, 32, 32, 7, 0, 1, 7),
    (512, 512, 512, 2, 0, 1, 2),
    (1024, 1024, 1024, 1, 0, 1, 1),
    (128, 384, 384, 3, 2, 3, 12),
    (128, 256, 64, 2, 0, 1, 2),
    (64, 256, 256, 5, 0, 1, 5),      # CTA pairs over 64-row slices; the last pair half past the end
    (256, 128, 128, 3, 1, 1, 5),     # CTA pairs with 128-column tiles (64 matrix rows per CTA)
]


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("R,C,Cout,batch,s0,ds,nslices", CASES)
def test_tc_slice_gemm(kind, R, C, Cout, batch, s0, ds, nslices):
    """kind 0: BF16 operands and output; 1: TF32 products, output rounded to TF32; 2: FP32 products
    formed from three TF32 products (about 2^-20 relative each), FP32 output."""
    g = torch.Generator(device="cuda").manual_seed(R * 7 + C + Cout + batch + kind)
    dt = torch.bfloat16 if kind == 0 else torch.float32
    X = torch.randn((nslices, R, C), device="cuda", generator=g).to(dt)
    Mat = torch.randn((C, Cout), device="cuda", generator=g).to(dt)
    MatT = Mat.t().contiguous()
    out = run(kind, X, s0, ds, batch, MatT).double()
    idx = torch.arange(batch, device="cuda") * ds + s0
    Xd = X[idx].double()
    Md = Mat.double()
    if kind == 1:  # TF32 keeps 10 explicit mantissa bits (kind 2 uses the FP32 values themselves)
        def tf32(t):
            i = t.float().view(torch.int32)
            return (i & ~0x1FFF).view(torch.float32).double()
        Xd, Md = tf32(X[idx]), tf32(Mat)
    ref = torch.matmul(Xd, Md).transpose(1, 2)
    scale = torch.matmul(Xd.abs(), Md.abs()).transpose(1, 2)
    if kind == 0:
        # output is rounded to BF16: 2^-8 relative, plus FP32 accumulation
        tol = 2.0 ** -8 * ref.abs() + 1e-5 * scale
    elif kind == 1:
        tol = 2e-3 * scale + 1e-6
    else:
        # three-product FP32: 2^-19 of each product, FP32 accumulation over C terms, FP32 output
        tol = (2.0 ** -19 + C * 2.0 ** -24) * scale + 2.0 ** -23 * ref.abs()
    bad = (out - ref).abs() > tol
    assert not bool(bad.any()), f"{int(bad.sum())} mismatches, max err {(out - ref).abs().max().item():.3e}"


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    """Failure detection in the allowed form: the tensor-core kernels' bounded mbarrier wait, given a
    1 ms limit, on a barrier nothing arrives at (no copy or product in flight), gives up, records its
    error code and returns; the library reports SFDE_ETIMEOUT and the context keeps working."""
    import ctypes as C
    import paper_1805_06688_gb300 as sfde
    from sfde_workloads import time_grid
    L = sfde.lib()
    L.sfde_debug_wait_timeout.argtypes = [C.c_ulonglong, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    err, waited = C.c_int(0), C.c_double(0.0)
    st = L.sfde_debug_wait_timeout(1000000, C.byref(err), C.byref(waited))
    assert st == sfde.SFDE_ETIMEOUT
    assert err.value == 1                      # the error code of a full-barrier wait
    assert 1e-3 <= waited.value < 0.5, waited.value
    assert L.sfde_debug_wait_timeout(10, None, None) == sfde.SFDE_EINVAL
    # the context is clean: a solve afterwards runs and converges
    P = sfde.Problem(0.7, 0.8, 1.0, 1.0, 16, 16, time_grid(32), precision=sfde.PREC_MIXED_BF16)
    P.set_initial(np.ones((16, 16)))
    _, stats = P.mgrit(m=4, rel_tol=1e-9, max_iter=40)
    assert stats.converged
    assert torch.cuda.is_available() and torch.zeros(4, device="cuda").sum().item() == 0.0
