"""Non-linear reaction r(u) = c u^p and Newton's method (Sec. 3) on the GPU
against the oracle: H and its Jacobian blocks element by element (through the
change of basis), and the Newton solution as a function, with its non-linear
residual measured by the oracle's operator."""
import numpy as np
import pytest

import oracle as O
from paper_1502_02941_gb300 import dg as D
from paper_1502_02941_gb300 import workloads as W
from gpu_helpers import basis_change, gpu_setup, oracle_run, x_to_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def _poly_u2(k, c=1.5):
    a, bb = {1: (1, 0), 2: (1, 1), 3: (2, 1)}[k]
    return W.Problem("poly_u2", 0.3, 0.7, (0.4, 0.3, -0.2, -0.6, 0.1, 0.5), W.polynomial(a, bb),
                     neumann_sides=("right", "top"), reaction=(2, c))


def _oracle_nonlinear_residual(run, xo, p, c):
    H, _ = O.nonlinear(run.mesh, run.k, xo, p, c)
    r = O.apply(run.mesh, run.system.A_diag, run.system.A_off, xo) + H - run.system.F
    return np.linalg.norm(r) / np.linalg.norm(run.system.F)


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("p", [2, 3])
def test_nonlinear_global_matches_oracle(k, p):
    """H(x) and the element blocks of its Jacobian: H_gpu(K) = T_K^T H_orc(K),
    HJ_gpu(K) = T_K^T HJ_orc(K) T_K, on a perturbed mesh with a ragged last
    tile (2 x 7^2 = 98 elements)."""
    ma = W.perturbed_mesh(7, seed=3)
    prob = _poly_u2(k)
    h = gpu_setup(ma, k, 2, prob)
    run = oracle_run(ma, k, 2, prob)
    T = basis_change(run, ma, k)
    nb = O.nbasis(k)
    rng = np.random.default_rng(100 * k + p)
    xg = rng.normal(size=ma.ne * nb)
    Hg, HJg = h.nonlinear_global(torch.tensor(xg, device="cuda"), p=p, c=0.8)
    Ho, HJo = O.nonlinear(run.mesh, k, x_to_oracle(T, xg), p, 0.8)
    Hexp = np.einsum("kmi,km->ki", T, Ho.reshape(ma.ne, nb)).reshape(-1)
    HJexp = np.einsum("kmi,kmn,knj->kij", T, HJo, T)
    np.testing.assert_allclose(_np(Hg), Hexp, rtol=0, atol=1e-12 * np.abs(Hexp).max())
    np.testing.assert_allclose(_np(HJg), HJexp, rtol=0, atol=1e-12 * np.abs(HJexp).max())
    h.close()


@pytest.mark.parametrize("method", [1, 2, 3])
def test_newton_on_the_papers_example_matches_oracle(method):
    """The paper's non-linear example (tanh layer, r(u) = u^2, 8x8 P1) for each
    method: the GPU Newton solution equals the oracle's as a function, and its
    non-linear residual measured with the oracle's operator is <= 1e-10."""
    c = W.tanh_nonlinear(method=method)
    ma = W.structured_mesh(c.N)
    h = gpu_setup(ma, c.k, c.method, c.problem, tol=1e-12, gmres_m=50)
    x, info = h.newton_solve(p=2, c=1.0, max_newton=30, lin_tol=1e-12)
    assert info.status == 0 and info.relres <= 1e-12 and 1 <= info.outer <= 15 and info.iterations > 0
    run = oracle_run(ma, c.k, c.method, c.problem)
    T = basis_change(run, ma, c.k)
    xo = x_to_oracle(T, _np(x))
    assert _oracle_nonlinear_residual(run, xo, 2, 1.0) <= 1e-10
    vo, steps, _ = O.newton(run.mesh, run.system, 2, 1.0, tol=1e-12)
    np.testing.assert_allclose(xo, vo, rtol=0, atol=1e-7 * np.abs(vo).max())
    # the paper's driver prints DoFs, h_max, L2 error and Newton steps
    from paper_1502_02941_gb300 import problem
    from helpers import oracle_l2
    l2g, hmax = h.l2_error(x, problem.exact_at_error_points(h, c.problem))
    l2o, hmo = oracle_l2(run, vo, c.problem)
    assert abs(l2g - l2o) <= 1e-8 * l2o and abs(hmax - hmo) <= 1e-15
    assert abs(info.outer - steps) <= 1
    h.close()


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("pc", ["bj", "schwarz"])
def test_newton_reproduces_polynomial_solutions(k, pc):
    """u in P_k with r(u) = 1.5 u^2: the GPU Newton solve reproduces it (L2 error
    of u_h), over several tiles with a ragged last one, with either
    preconditioner set up on the Jacobian; a linear solve afterwards sets the
    preconditioner up on A again and solves A x = F."""
    from paper_1502_02941_gb300 import problem
    prob = _poly_u2(k)
    ma = W.perturbed_mesh(9, seed=7, neumann_sides=prob.neumann_sides)   # 162 elements
    prec = D.DG_PRECOND_SCHWARZ if pc == "schwarz" else D.DG_PRECOND_BLOCK_JACOBI
    h = gpu_setup(ma, k, 2, prob, tol=1e-12, gmres_m=30, precond=prec)
    x, info = h.newton_solve(p=2, c=1.5, max_newton=20, lin_tol=1e-12)
    assert info.status == 0 and info.relres <= 1e-12
    l2, _ = h.l2_error(x, problem.exact_at_error_points(h, prob))
    assert l2 < 1e-9
    xl, _ = h.gmres_solve()
    run = oracle_run(ma, k, 2, prob)
    T = basis_change(run, ma, k)
    xo = x_to_oracle(T, _np(xl))
    r = run.system.F - O.apply(run.mesh, run.system.A_diag, run.system.A_off, xo)
    assert np.linalg.norm(r) / np.linalg.norm(run.system.F) <= 1e-10
    h.close()


def test_newton_argument_errors():
    c = W.tanh_nonlinear()
    ma = W.structured_mesh(c.N)
    h = gpu_setup(ma, c.k, c.method, c.problem)
    for kw in ({"p": 0}, {"p": 5}, {"max_newton": 0}, {"lin_tol": 1.0}):
        with pytest.raises(D.DGError) as e:
            h.newton_solve(**kw)
        assert e.value.status == D.DG_ERR_INVALID_ARG
    h.set_params(precond=D.DG_PRECOND_MLP)
    with pytest.raises(D.DGError) as e:
        h.newton_solve()
    assert e.value.status == D.DG_ERR_INVALID_ARG
    h.close()
