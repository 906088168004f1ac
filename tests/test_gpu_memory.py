"""The handle's device memory (include/dg.h, "device memory of a handle"):
per-category sizes from dg_workspace_size, and the two caller-supplied memory
sources -- a caller arena (a torch-allocated buffer) and a caller allocator
(torch's caching allocator through ctypes callbacks).  A handle on either
source gives the same solutions as a handle on cudaMalloc, holds all of its
device memory there, and reports exhaustion as DG_ERR_NOMEM."""
import numpy as np
import pytest

from paper_1502_02941_gb300 import dg as D
from paper_1502_02941_gb300 import problem
from paper_1502_02941_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CATS = (D.DG_WS_MESH, D.DG_WS_OPERATOR, D.DG_WS_PRECOND, D.DG_WS_SOLVER, D.DG_WS_LEARNED, D.DG_WS_SCRATCH)


def _pipeline(h):
    """Mesh, f64 + f32 assembly, Schwarz set-up, f64 GMRES, f32-refined solve,
    L2 error: the calls that allocate for one workload (32x32 P2 boundary layer)."""
    cfg = W.boundary_layer_p2(method=1, N=32)
    problem.setup(h, cfg, store=D.DG_STORE_F64 | D.DG_STORE_F32, gmres_m=30, tol=1e-10, max_it=20000,
                  precond=D.DG_PRECOND_SCHWARZ)
    h.precond_setup(D.DG_PRECOND_SCHWARZ)
    x64, _ = h.gmres_solve()
    x32, _ = h.mixed_solve(D.DG_F32, inner_m=30, inner_tol=1e-3, max_outer=40)
    l2, _ = h.l2_error(x64, problem.exact_at_error_points(h, cfg.problem))
    torch.cuda.synchronize()
    return x64.cpu().numpy(), x32.cpu().numpy(), l2


def _sizes(h):
    return {c: h.workspace_size(c) for c in (D.DG_WS_TOTAL, *CATS, D.DG_WS_PEAK)}


def test_workspace_sizes_by_category():
    h = D.DG(0)
    ref = _pipeline(h)
    sz = _sizes(h)
    info = h.info()
    assert sz[D.DG_WS_TOTAL] == sum(sz[c] for c in CATS)
    assert sz[D.DG_WS_PEAK] >= sz[D.DG_WS_TOTAL] > 0
    for c in (D.DG_WS_MESH, D.DG_WS_OPERATOR, D.DG_WS_PRECOND, D.DG_WS_SOLVER, D.DG_WS_SCRATCH):
        assert sz[c] > 0, c
    assert sz[D.DG_WS_LEARNED] == 0
    # the operator category is exactly the stored block copies and F
    assert sz[D.DG_WS_OPERATOR] == sum(info.block_bytes) + 8 * info.dofs
    # the Krylov basis of the f64 GMRES(30) alone: 32 vectors of the padded length
    assert sz[D.DG_WS_SOLVER] >= 32 * 8 * info.dofs
    h.close()
    assert D.dg_workspace_size(None, D.DG_WS_TOTAL) == 0
    assert ref[2] > 0


def test_arena_from_a_torch_buffer():
    h = D.DG(0)
    ref = _pipeline(h)
    peak = h.workspace_size(D.DG_WS_PEAK)
    h.close()
    # an arena of the reported peak plus a quarter: same results, all memory inside
    buf = torch.empty(int(peak * 1.25) + (1 << 20), dtype=torch.uint8, device="cuda")
    ha = D.DG(0)
    ha.set_arena(buf)
    got = _pipeline(ha)
    for a, b in zip(ref[:2], got[:2]):
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-13 * np.abs(a).max())
    assert abs(got[2] - ref[2]) <= 1e-13 * ref[2]
    assert 0 < ha.workspace_size(D.DG_WS_TOTAL) <= buf.numel()
    ha.close()
    # a second source after memory was taken is refused; a small arena runs out cleanly
    hs = D.DG(0)
    hs.set_arena(buf[: 1 << 16])
    with pytest.raises(D.DGError) as e:
        _pipeline(hs)
    assert e.value.status == D.DG_ERR_NOMEM
    with pytest.raises(D.DGError) as e:
        hs.set_arena(buf)
    assert e.value.status == D.DG_ERR_STATE
    hs.close()
    # host memory and misaligned bases are refused
    hb = D.DG(0)
    with pytest.raises(ValueError):
        hb.set_arena(buf.cpu())
    assert D.dg_set_arena(hb.h, buf.data_ptr() + 8, 1 << 20) == D.DG_ERR_INVALID_ARG
    hb.close()


def test_torch_caching_allocator_as_the_memory_source():
    h = D.DG(0)
    ref = _pipeline(h)
    h.close()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    ht = D.DG(0)
    ht.use_torch_allocator()
    got = _pipeline(ht)
    held = ht.workspace_size(D.DG_WS_TOTAL)
    n_arrays = 64                       # far more than the handle's live arrays
    grown_open = torch.cuda.memory_allocated() - base
    for a, b in zip(ref[:2], got[:2]):
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-13 * np.abs(a).max())
    ht.close()
    torch.cuda.synchronize()
    grown_closed = torch.cuda.memory_allocated() - base
    # what the handle gave back to torch is what it reported holding, up to
    # torch's rounding of each array to 512-byte blocks
    released = grown_open - grown_closed
    assert held <= released <= held + 512 * n_arrays, (held, released)
