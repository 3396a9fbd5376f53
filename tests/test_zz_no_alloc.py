"""sfde_step_batch_noalloc against sfde_step_batch, through the C ABI.

The no-allocation entry point serves callers that cannot let the library call cudaMalloc or
cudaFree (device memory owned by another allocator, latency-critical loops where cudaFree would
synchronise the device).  It must give the same result as the allocating entry point, on two calls
in a row (the second call reuses the fixed scratch that the first one left behind), and refuse a
request larger than its fixed scratch before doing any work.  This file is collected last.
"""
import numpy as np
import pytest

from sfde_workloads import gaussian_bump_forcing, time_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_06688_gb300 as sfde  # noqa: E402


def _reldiff(a, b):
    return float((a - b).abs().max() / b.abs().max())


def test_noalloc_step_matches_allocating_step_twice():
    nx, ny, nt = 50, 70, 24
    t = time_grid(nt, 1.0, "graded")
    F, _ = gaussian_bump_forcing(3, nx, ny, t)
    P = sfde.Problem(0.7, 0.85, 1.3, 0.4, nx, ny, t)
    P.set_forcing(F)
    g = torch.Generator(device="cuda").manual_seed(11)
    for call, (n0, dn, batch) in enumerate([(2, 4, 6), (1, 3, 8)]):
        src = torch.randn((batch, ny, nx), dtype=torch.float64, device="cuda", generator=g)
        ref = torch.empty_like(src)
        P.step_batch(n0, dn, src, ref)
        out = torch.full_like(src, float("nan"))
        st = sfde.sfde_step_batch_noalloc(P.ctx, n0, dn, batch, src, out)
        assert st == sfde.SFDE_OK, sfde.sfde_strerror(st)
        torch.cuda.synchronize()
        # same kernels and operation order: equal to the tolerance of the step parity tests
        assert _reldiff(out, ref) < 1e-11, (call, _reldiff(out, ref))


def test_noalloc_rejects_requests_beyond_the_scratch():
    n, nt = 255, 8                         # padded extent 256: 5 * batch * 256^2 doubles needed
    P = sfde.Problem(0.6, 0.9, 1.0, 0.5, n, n, time_grid(nt))
    limit_batch = sfde.NOALLOC_SCRATCH_DOUBLES // (5 * 256 * 256)
    src = torch.zeros((limit_batch + 1, n, n), dtype=torch.float64, device="cuda")
    out = torch.zeros_like(src)
    st = sfde.sfde_step_batch_noalloc(P.ctx, 1, 1, limit_batch + 1, src, out)
    assert st == sfde.SFDE_ESCRATCH
    # host buffers are refused (the entry point never stages through a temporary device copy): by
    # the binding before the call, and by the C entry point itself
    host = np.zeros((1, n, n))
    with pytest.raises(ValueError):
        sfde.sfde_step_batch_noalloc(P.ctx, 1, 1, 1, host, host.copy())
    host2 = host.copy()
    assert sfde.lib().sfde_step_batch_noalloc(P.ctx, 1, 1, 1, host.ctypes.data, host2.ctypes.data) == sfde.SFDE_EINVAL
    # a batch larger than the tensors hold is refused by the binding
    with pytest.raises(ValueError):
        sfde.sfde_step_batch_noalloc(P.ctx, 1, 1, 2, src[:1], out[:1])
    # at the limit it runs
    ok = sfde.sfde_step_batch_noalloc(P.ctx, 1, 1, limit_batch, src[:limit_batch], out[:limit_batch])
    assert ok == sfde.SFDE_OK
    torch.cuda.synchronize()
