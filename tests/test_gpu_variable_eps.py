"""A variable diffusion coefficient eps(x, y) (the paper's fdiff, Sec. 2.2)
on the GPU against the oracle: the face point set, the assembled blocks and F
element by element (1e-11, as the constant-eps parity tests), the rounded
low-precision copies, P_k reproduction with an affine eps, a GMRES solution,
and the argument checks."""
import numpy as np
import pytest

import oracle as O
from paper_1502_02941_gb300 import dg as D
from paper_1502_02941_gb300 import problem
from paper_1502_02941_gb300 import workloads as W
from gpu_helpers import (basis_change, gpu_setup, oracle_blocks, oracle_run, rel_residual_oracle, to_gpu_basis,
                         x_to_oracle)
from helpers import oracle_direct, oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def _rel_close(a, b, tol):
    scale = np.abs(b).max()
    err = np.abs(a - b).max()
    assert err <= tol * scale, (err, scale, err / scale)


def _wavy_problem():
    return W.Problem("gauss", 0.0, 0.4, (0.5, 0.0, -1.0, -0.5, 1.0, 0.0), W.gaussian_bump,
                     neumann_sides=("right", "top"), eps_fn=W.wavy_eps(0.05, 0.03))


def test_face_points_match_the_oracle_edge_points():
    ma = W.perturbed_mesh(4, seed=1, neumann_sides=("right",))
    k = 2
    h = D.DG(0)
    h.mesh_upload(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
    h.set_params(degree=k)
    xf = _np(h.quad_points(D.DG_POINTS_FACE))                 # [ne, 3, k+2, 2]
    m = O.make_mesh(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
    xe = O.quad_points(m, k, O.EDGES)                          # [ned, k+2, 2]
    for K in range(ma.ne):
        for f in range(3):
            e = m.elem_edges[K, f]
            g = sorted(map(tuple, xf[K, f].round(12)))
            o = sorted(map(tuple, xe[e].round(12)))
            assert g == o
            # each face runs from local vertex f to f+1
            a, b = ma.nodes[ma.elems[K, f]], ma.nodes[ma.elems[K, (f + 1) % 3]]
            t = np.linalg.norm(xf[K, f] - a, axis=1) / np.linalg.norm(b - a)
            assert np.all(np.diff(t) > 0)
    h.close()


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("method", [1, 2, 3])
def test_variable_eps_assembly_parity(k, method):
    prob = _wavy_problem()
    ma = W.perturbed_mesh(5, seed=11, neumann_sides=prob.neumann_sides)
    h = gpu_setup(ma, k, method, prob, store=D.DG_STORE_F64 | D.DG_STORE_F32 | D.DG_STORE_BF16)
    Ag, _ = h.blocks()
    Fg = _np(h.rhs())
    run = oracle_run(ma, k, method, prob)
    T = basis_change(run, ma, k)
    Ao, nbr = oracle_blocks(run, ma)
    _rel_close(_np(Ag), to_gpu_basis(T, Ao, nbr), 1e-11)
    _rel_close(Fg, np.einsum("kmi,km->ki", T, run.system.F.reshape(ma.ne, -1)).reshape(-1), 1e-11)
    # the low-precision copies are the rounded f64 blocks
    A64 = _np(Ag)
    for dt, tol in ((D.DG_F32, 2 ** -24), (D.DG_BF16, 2 ** -8)):
        Alo = _np(h.blocks(dt)[0].double())
        assert np.all(np.abs(Alo - A64) <= tol * np.abs(A64) + 1e-300)
    h.close()


def test_variable_eps_superpenalised_assembly_parity():
    prob = _wavy_problem()
    ma = W.perturbed_mesh(4, seed=3, neumann_sides=prob.neumann_sides)
    h = gpu_setup(ma, 2, 2, prob, b0=2.5)
    run = oracle_system(ma, 2, 2, prob, b0=2.5)
    T = basis_change(run, ma, 2)
    Ao, nbr = oracle_blocks(run, ma)
    _rel_close(_np(h.blocks()[0]), to_gpu_basis(T, Ao, nbr), 1e-11)
    _rel_close(_np(h.rhs()), np.einsum("kmi,km->ki", T, run.system.F.reshape(ma.ne, -1)).reshape(-1), 1e-11)
    h.close()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_variable_eps_polynomial_reproduction_gpu(k):
    """Affine eps(x, y) = 0.5 + 0.3 x - 0.2 y and u in P_k: all three methods
    reproduce u through the GPU assembly and GMRES (the method's consistency,
    independent of the oracle)."""
    a, bb = {1: (1, 0), 2: (1, 1), 3: (2, 1)}[k]
    prob = W.Problem("poly", 0.0, 0.7, (0.4, 0.3, -0.2, -0.6, 0.1, 0.5), W.polynomial(a, bb),
                     neumann_sides=("right", "top"), eps_fn=W.affine_eps(0.5, 0.3, -0.2))
    ma = W.perturbed_mesh(4, seed=7, neumann_sides=prob.neumann_sides)
    for method in (1, 2, 3):
        h = gpu_setup(ma, k, method, prob, tol=1e-13, gmres_m=30)
        xg, info = h.gmres_solve()
        l2, _ = h.l2_error(xg, problem.exact_at_error_points(h, prob))
        assert l2 < 1e-10, (method, l2, info.relres)
        h.close()


def test_variable_eps_gmres_solution_matches_oracle():
    prob = W.Problem("sinsin", 0.0, 0.2, (0.3, 0.0, 0.0, -0.2, 0.0, 0.0), W.sinsin, eps_fn=W.wavy_eps(1.0, 0.5))
    ma = W.structured_mesh(12)
    h = gpu_setup(ma, 2, 2, prob, tol=1e-12, gmres_m=30)
    xg, info = h.gmres_solve()
    assert info.status == D.DG_OK
    run = oracle_run(ma, 2, 2, prob)
    T = basis_change(run, ma, 2)
    assert rel_residual_oracle(run, T, _np(xg)) <= 1e-10
    xo = oracle_direct(run)
    assert np.abs(x_to_oracle(T, _np(xg)) - xo).max() <= 1e-8 * np.abs(xo).max()
    h.close()


def test_variable_eps_argument_checks():
    prob = _wavy_problem()
    ma = W.perturbed_mesh(3, seed=2, neumann_sides=prob.neumann_sides)
    h = D.DG(0)
    cfg = W.Config("t", 0, 2, 2, prob)
    problem.setup(h, cfg, mesh=ma, assemble=False)
    data = problem.problem_data(h, prob)
    eq, ef = problem.eps_data(h, prob)
    with pytest.raises(D.DGError) as e:                      # eps_q without eps_f
        h.assemble(0.0, prob.alpha, prob.b, *data, eps_q=eq)
    assert e.value.status == D.DG_ERR_INVALID_ARG
    h.set_params(store=D.DG_STORE_F32)
    with pytest.raises(D.DGError) as e:                      # no f64 copy to add into
        h.assemble(0.0, prob.alpha, prob.b, *data, eps_q=eq, eps_f=ef)
    assert e.value.status == D.DG_ERR_INVALID_ARG
    with pytest.raises(ValueError):                          # binding: too few entries
        h.assemble(0.0, prob.alpha, prob.b, *data, eps_q=eq, eps_f=ef[:-1].contiguous())
    h.set_params(store=D.DG_STORE_F64)
    h.batch_setup(np.array([0, ma.ne], np.int32), np.array([[0.05, prob.alpha, *prob.b]]))
    with pytest.raises(D.DGError) as e:                      # batch mode reads per-instance constants
        h.assemble(0.0, prob.alpha, prob.b, *data, eps_q=eq, eps_f=ef)
    assert e.value.status == D.DG_ERR_INVALID_ARG
    h.close()
