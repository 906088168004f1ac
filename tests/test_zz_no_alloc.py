"""The allocation-free L2-error entry point (dg_l2_error_noalloc) against the
regular dg_l2_error, through the C ABI.

dg_l2_error_noalloc serves callers that cannot allocate device memory (all of
it owned by another allocator, or a timing-critical loop that must not call
cudaMalloc); its scratch is a fixed array inside the library.  This
file is collected last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1502_02941_gb300 import dg as D
from paper_1502_02941_gb300 import problem
from paper_1502_02941_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_l2_error_noalloc_matches_regular_entry_point():
    cfg = W.boundary_layer_p2(method=2, N=24)          # 1152 triangles, P2
    h = D.DG(0)
    problem.setup(h, cfg, tol=1e-12)
    x, _ = h.gmres_solve()
    uex = problem.exact_at_error_points(h, cfg.problem)
    l2_ref, hmax_ref = h.l2_error(x, uex)
    # two calls in a row on the same data, then one on different data
    for _ in range(2):
        s, l2, hmax = D.dg_l2_error_noalloc(h.h, x, uex)
        assert s == D.DG_OK, D.dg_last_error(h.h)
        assert abs(l2 - l2_ref) <= 1e-12 * l2_ref
        assert hmax == hmax_ref
    x2 = (0.5 * x).contiguous()
    l2_ref2, _ = h.l2_error(x2, uex)
    s, l2b, _ = D.dg_l2_error_noalloc(h.h, x2, uex)
    assert s == D.DG_OK and abs(l2b - l2_ref2) <= 1e-12 * l2_ref2
    h.close()


def test_l2_error_noalloc_binding_checks_sizes_and_memory_kind():
    cfg = W.boundary_layer_p2(method=2, N=4)
    h = D.DG(0)
    problem.setup(h, cfg)
    info = h.info()
    uex = problem.exact_at_error_points(h, cfg.problem)
    x = torch.zeros(info.dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        D.dg_l2_error_noalloc(h.h, x.cpu().numpy(), uex)            # host array as device memory
    with pytest.raises(ValueError):
        D.dg_l2_error_noalloc(h.h, x[:-1], uex)                      # one entry short
    with pytest.raises(ValueError):
        D.dg_l2_error_noalloc(h.h, x.float(), uex)                   # f32 where f64 is read
    s, l2, _ = D.dg_l2_error_noalloc(h.h, x, uex)
    assert s == D.DG_OK and l2 > 0
    h.close()


def test_l2_error_noalloc_rejects_oversized_mesh():
    ma = W.structured_mesh(1449)             # 4,199,202 triangles > 4,194,304
    h = D.DG(0)
    h.mesh_upload(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
    h.set_params(degree=1)
    h.boundary_info()                        # builds the reference tables
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    # the binding would refuse a 16-entry buffer for this mesh; raw addresses
    # reach the library, whose own size bound must reject the call before any
    # launch (nothing is read from the buffer)
    s, _, _ = D.dg_l2_error_noalloc(h.h, dummy.data_ptr(), dummy.data_ptr())
    assert s == D.DG_ERR_INVALID_ARG
    assert "4194304" in D.dg_last_error(h.h)
    h.close()
