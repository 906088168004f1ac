"""Host-side fault injection on a GPU handle (no GPU fault is involved): a
forced CUDA runtime error maps to DG_ERR_CUDA with the failing call named,
and the handle stays usable; a caller allocator that returns NULL maps to
DG_ERR_NOMEM."""
import numpy as np
import pytest

from paper_1502_02941_gb300 import dg as D
from paper_1502_02941_gb300 import problem
from paper_1502_02941_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solve(h, cfg):
    problem.setup(h, cfg, tol=1e-11, gmres_m=30)
    x, info = h.gmres_solve()
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


@pytest.mark.parametrize("n", [1, 4, 12])
def test_injected_cuda_error_maps_to_dg_err_cuda(monkeypatch, n):
    cfg = W.sine_8x8()
    ref = D.DG(0)
    x_ref, _ = _solve(ref, cfg)
    ref.close()
    monkeypatch.setenv("DG_FAIL_CUDA_CALL", str(n))
    h = D.DG(0)                                 # the hook is read at dg_create
    monkeypatch.delenv("DG_FAIL_CUDA_CALL")
    with pytest.raises(D.DGError) as e:
        _solve(h, cfg)
    assert e.value.status == D.DG_ERR_CUDA
    assert "injected failure" in str(e.value)
    # the same handle runs the whole sequence again and gets the clean result
    x, info = _solve(h, cfg)
    assert info.status == D.DG_OK
    np.testing.assert_allclose(x, x_ref, rtol=0, atol=1e-12 * np.abs(x_ref).max())
    h.close()


def test_caller_allocator_returning_null_maps_to_dg_err_nomem():
    h = D.DG(0)
    calls = []

    def alloc(ctx, nbytes, device, stream):
        calls.append(nbytes)
        return None                              # out of memory

    def free(ctx, ptr, nbytes, device, stream):
        pass

    fns = (D.DG_ALLOC_FN(alloc), D.DG_FREE_FN(free))
    assert D.dg_set_allocator(h.h, *fns) == D.DG_ERR_NOMEM     # the 64-byte flag block already fails
    assert calls == [64]
    # the handle stayed on cudaMalloc and works
    x, info = _solve(h, W.sine_8x8())
    assert info.status == D.DG_OK and h.workspace_size(D.DG_WS_TOTAL) > 0
    h.close()
