"""GPU parity: every libdg call against the FP64 CPU oracle on the same seeded
inputs (element by element, through the change of basis), plus pins that hold
without the oracle (polynomial reproduction, SIPG symmetry).

Tolerances: the FP64 path is compared entry by entry at 1e-11 relative to the
largest entry of the compared object (rounding of O(100)-term sums and of the
basis change; the method fixes the result exactly); solutions as functions at
1e-10 after a direct solve.  f32 / bf16 applies are compared with the same
stored low-precision blocks evaluated in f64 (accumulation error only) and the
stored blocks with the f64 blocks (rounding error only).
"""
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


def _poly_problem(k, neumann=("right", "top")):
    a, bb = {1: (1, 0), 2: (1, 1), 3: (2, 1)}[k]
    return W.Problem("poly", 0.3, 0.7, (0.4, 0.3, -0.2, -0.6, 0.1, 0.5), W.polynomial(a, bb),
                     neumann_sides=neumann)


def _bumpy_problem():
    return W.Problem("gauss", 0.05, 0.4, (0.5, 0.0, -1.0, -0.5, 1.0, 0.0), W.gaussian_bump,
                     neumann_sides=("right", "top"))


def _np(t):
    return t.detach().cpu().numpy()


# ----------------------------------------------------------------------------
# mesh
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("which", ["fixture", "perturbed"])
def test_adjacency_matches_oracle(which):
    if which == "fixture":
        ma = W.MeshArrays(W.FIXTURE_NODES, W.FIXTURE_ELEMS, W.FIXTURE_DIRICHLET, np.zeros((0, 2), np.int32))
    else:
        ma = W.perturbed_mesh(5, seed=3, neumann_sides=("top", "left"))
    h = D.DG(0)
    h.mesh_upload(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
    h.set_params(degree=1)
    info = h.info()
    m = O.make_mesh(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
    assert info.ne == m.ne and info.n_bedges == m.n_bedges and info.n_interior == m.n_interior
    h.assemble(1.0, 0.0, (0,) * 6)
    _, nbr = h.blocks()
    nbr = _np(nbr)
    for K in range(m.ne):
        for f in range(3):
            va, vb, Ki, Kj, typ = m.edges[m.elem_edges[K, f]]
            exp = -1 if Kj < 0 else (Kj if Ki == K else Ki)
            assert nbr[K, f] == exp
    # boundary numbering: (element, face) order; type and outward normal agree
    nrm, typ = h.boundary_info()
    nrm, typ = _np(nrm), _np(typ)
    bfaces = [(K, f) for K in range(m.ne) for f in range(3) if nbr[K, f] < 0]
    assert len(bfaces) == info.n_bedges
    onrm, otyp = O.boundary_normals(m), O.boundary_types(m)
    be = np.where(m.edges[:, 3] < 0)[0]
    pos = {int(e): i for i, e in enumerate(be)}
    for b, (K, f) in enumerate(bfaces):
        i = pos[int(m.elem_edges[K, f])]
        assert typ[b] == otyp[i]
        np.testing.assert_allclose(nrm[b], onrm[i], atol=1e-15)
    h.close()


def test_mesh_errors_are_reported():
    ma = W.structured_mesh(3)
    h = D.DG(0)
    bad = ma.elems.copy()
    bad[4] = bad[4, ::-1]
    with pytest.raises(D.DGError) as e:
        h.mesh_upload(ma.nodes, bad, ma.dirichlet, ma.neumann)
    assert e.value.status == D.DG_ERR_MESH
    with pytest.raises(D.DGError) as e:
        h.mesh_upload(ma.nodes, ma.elems, ma.dirichlet[:-1], ma.neumann)
    assert e.value.status == D.DG_ERR_MESH
    interior_edge = np.array([[ma.elems[0, 0], ma.elems[0, 2]]], np.int32)   # the "/" diagonal
    with pytest.raises(D.DGError) as e:
        h.mesh_upload(ma.nodes, ma.elems, np.concatenate([ma.dirichlet, interior_edge]), ma.neumann)
    assert e.value.status == D.DG_ERR_MESH
    bad_idx = ma.elems.copy()
    bad_idx[0, 0] = 10 ** 6
    with pytest.raises(D.DGError) as e:
        h.mesh_upload(ma.nodes, bad_idx, ma.dirichlet, ma.neumann)
    assert e.value.status == D.DG_ERR_MESH
    with pytest.raises(D.DGError) as e:
        h.apply(torch.zeros(10, dtype=torch.float64, device="cuda"))
    assert e.value.status == D.DG_ERR_STATE
    h.close()


@pytest.mark.parametrize("k", [1, 3])
def test_quadrature_points_match_oracle(k):
    ma = W.perturbed_mesh(4, seed=1, neumann_sides=("right",))
    h = D.DG(0)
    h.mesh_upload(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
    h.set_params(degree=k)
    m = O.make_mesh(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
    for which, ow in ((D.DG_POINTS_VOLUME, O.VOLUME), (D.DG_POINTS_ERROR, O.ERROR)):
        g = np.sort(_np(h.quad_points(which)).round(12).view("f8,f8"), axis=1)
        o = np.sort(O.quad_points(m, k, ow).round(12).view("f8,f8"), axis=1)
        assert np.array_equal(g, o)
    # boundary points: each GPU boundary edge carries the oracle's point set
    gb = _np(h.quad_points(D.DG_POINTS_BOUNDARY))
    ob = O.quad_points(m, k, O.BOUNDARY)
    gset = sorted(tuple(sorted(map(tuple, e.round(12)))) for e in gb)
    oset = sorted(tuple(sorted(map(tuple, e.round(12)))) for e in ob)
    assert gset == oset
    h.close()


# ----------------------------------------------------------------------------
# assembly, RHS, apply, block Jacobi
# ----------------------------------------------------------------------------


def _rel_close(a, b, tol):
    scale = np.abs(b).max()
    err = np.abs(a - b).max()
    assert err <= tol * scale, (err, scale, err / scale)


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("method", [1, 2, 3])
def test_assembly_parity(k, method):
    prob = _bumpy_problem()
    ma = W.perturbed_mesh(5, seed=11, neumann_sides=prob.neumann_sides)
    h = gpu_setup(ma, k, method, prob)
    Ag, _ = h.blocks()
    Fg = _np(h.rhs())
    run = oracle_run(ma, k, method, prob)
    T = basis_change(run, ma, k)
    Ao, nbr = oracle_blocks(run, ma)
    Ao_g = to_gpu_basis(T, Ao, nbr)
    _rel_close(_np(Ag), Ao_g, 1e-11)
    Fo_g = np.einsum("kmi,km->ki", T, run.system.F.reshape(ma.ne, -1)).reshape(-1)
    _rel_close(Fg, Fo_g, 1e-11)
    h.close()


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("method", [1, 2])
def test_superpenalised_assembly_parity(k, method):
    """Superpenalisation b0 = 2.5 (penalty sigma eps / |e|^b0): blocks and F
    equal the oracle's, and b0 outside [1, 8] is refused."""
    prob = _bumpy_problem()
    ma = W.perturbed_mesh(5, seed=11, neumann_sides=prob.neumann_sides)
    h = gpu_setup(ma, k, method, prob, b0=2.5)
    Ag, _ = h.blocks()
    Fg = _np(h.rhs())
    run = oracle_system(ma, k, method, prob, b0=2.5)
    T = basis_change(run, ma, k)
    Ao, nbr = oracle_blocks(run, ma)
    _rel_close(_np(Ag), to_gpu_basis(T, Ao, nbr), 1e-11)
    _rel_close(Fg, np.einsum("kmi,km->ki", T, run.system.F.reshape(ma.ne, -1)).reshape(-1), 1e-11)
    with pytest.raises(D.DGError) as e:
        h.set_params(b0=0.5)
    assert e.value.status == D.DG_ERR_INVALID_ARG
    h.close()


def test_sipg_symmetric_on_gpu():
    """b = 0, SIPG: the assembled GPU operator is symmetric (basis change by an
    element-wise T preserves symmetry)."""
    prob = W.Problem("s", 1.0, 0.3, (0,) * 6, W.sinsin)
    ma = W.perturbed_mesh(4, seed=2)
    h = gpu_setup(ma, 2, 2, prob)
    A, nbr = h.blocks()
    A, nbr = _np(A), _np(nbr)
    scale = np.abs(A).max()
    for K in range(ma.ne):
        assert np.abs(A[K, 0] - A[K, 0].T).max() <= 1e-14 * scale
        for f in range(3):
            L = nbr[K, f]
            if L < 0:
                continue
            g = list(nbr[L]).index(K)
            assert np.abs(A[K, 1 + f] - A[L, 1 + g].T).max() <= 1e-14 * scale
    h.close()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_apply_parity(k):
    prob = _bumpy_problem()
    ma = W.perturbed_mesh(6, seed=5, neumann_sides=prob.neumann_sides)
    h = gpu_setup(ma, k, 1, prob, store=D.DG_STORE_F64 | D.DG_STORE_F32 | D.DG_STORE_BF16)
    run = oracle_run(ma, k, 1, prob)
    T = basis_change(run, ma, k)
    nb = O.nbasis(k)
    rng = np.random.default_rng(k)
    xg = rng.standard_normal(ma.ne * nb)
    xt = torch.tensor(xg, device="cuda")
    yg = _np(h.apply(xt, D.DG_F64))
    yo = O.apply(run.mesh, run.system.A_diag, run.system.A_off, x_to_oracle(T, xg))
    yo_g = np.einsum("kmi,km->ki", T, yo.reshape(ma.ne, nb)).reshape(-1)
    # through the basis change (conditioning of T for P3 monomials ~1e4): 1e-11
    _rel_close(yg, yo_g, 1e-11)
    # f32 / bf16: same stored blocks in f64 (accumulation error), stored vs f64 blocks (rounding)
    A64, nbr = h.blocks(D.DG_F64)
    A64, nbr = _np(A64), _np(nbr)

    def ref_apply(A, x):
        X = x.reshape(ma.ne, nb)
        y = np.einsum("kij,kj->ki", A[:, 0], X)
        for f in range(3):
            L = nbr[:, f]
            ok = L >= 0
            y[ok] += np.einsum("kij,kj->ki", A[ok, 1 + f], X[L[ok]])
        return y.reshape(-1)

    np.testing.assert_allclose(ref_apply(A64, xg), yg, rtol=0, atol=1e-13 * np.abs(yg).max())
    for dt, tdt, acc_tol, round_tol in ((D.DG_F32, torch.float32, 2e-6, 2 ** -24), (D.DG_BF16, torch.bfloat16, 2e-6, 2 ** -8)):
        Alo, _ = h.blocks(dt)
        Alo = _np(Alo.double())
        assert np.all(np.abs(Alo - A64) <= round_tol * np.abs(A64) + 1e-300)
        x32 = xt.float()
        ylo = _np(h.apply(x32, dt).double())
        yref = ref_apply(Alo, _np(x32.double()))
        assert np.abs(ylo - yref).max() <= acc_tol * np.abs(yref).max()
    h.close()


@pytest.mark.parametrize("k", [1, 3])
def test_block_jacobi_parity(k):
    prob = _bumpy_problem()
    ma = W.perturbed_mesh(4, seed=8, neumann_sides=prob.neumann_sides)
    h = gpu_setup(ma, k, 2, prob)
    h.precond_setup()
    run = oracle_run(ma, k, 2, prob)
    T = basis_change(run, ma, k)
    inv_o = O.block_jacobi(run.system.A_diag)
    nb = O.nbasis(k)
    r = np.random.default_rng(0).standard_normal(ma.ne * nb)
    zg = _np(h.precond_apply(torch.tensor(r, device="cuda"), D.DG_F64))
    # z_gpu = T^-1 inv_o T^-T r
    R = r.reshape(ma.ne, nb)
    u = np.linalg.solve(np.transpose(T, (0, 2, 1)), R[..., None])[..., 0]
    v = np.einsum("kmn,kn->km", inv_o, u)
    zo = np.linalg.solve(T, v[..., None])[..., 0].reshape(-1)
    _rel_close(zg, zo, 1e-10)
    z32 = _np(h.precond_apply(torch.tensor(r, device="cuda", dtype=torch.float32), D.DG_F32).double())
    _rel_close(z32, zo, 1e-5)
    h.close()


def test_singular_block_reported():
    """alpha = eps = 0, b = 0 makes every diagonal block zero."""
    ma = W.structured_mesh(2)
    h = gpu_setup(ma, 1, 2, W.Problem("z", 0.0, 0.0, (0,) * 6, W.sinsin))
    with pytest.raises(D.DGError) as e:
        h.precond_setup()
    assert e.value.status == D.DG_ERR_SINGULAR_BLOCK
    h.close()


# ----------------------------------------------------------------------------
# solves, L2 error, evaluation
# ----------------------------------------------------------------------------


def test_sine_8x8_dense_solve_and_l2():
    cfg = W.sine_8x8()
    ma = W.structured_mesh(cfg.N)
    h = gpu_setup(ma, cfg.k, cfg.method, cfg.problem, sigma=cfg.sigma)
    xg = h.dense_solve()
    l2g, hmax = h.l2_error(xg, problem.exact_at_error_points(h, cfg.problem))
    run = oracle_run(ma, cfg.k, cfg.method, cfg.problem, sigma=cfg.sigma)
    xo = oracle_direct(run)
    T = basis_change(run, ma, cfg.k)
    xg_o = x_to_oracle(T, _np(xg))
    assert np.abs(xg_o - xo).max() <= 1e-10 * np.abs(xo).max()
    xe = O.quad_points(run.mesh, cfg.k, O.ERROR)
    l2o, hmo = O.l2_error(run.mesh, cfg.k, xo, cfg.problem.u(np, xe[..., 0], xe[..., 1]))
    assert abs(l2g - l2o) <= 1e-10 * l2o and abs(hmax - hmo) <= 1e-15
    h.close()


@pytest.mark.parametrize("method", [1, 2, 3])
def test_papers_linear_example(method):
    """The paper's linear example (Sec. 2: tanh internal layer, eps = 1e-6,
    b = (1,2)/sqrt(5), alpha = 1, P1 on the twice-refined initial mesh): the
    dense and the GMRES solve equal the oracle's direct solve as functions, and
    the L2 error and h_max its dg_error."""
    c = W.tanh_nonlinear(method=method)
    prob = W.Problem("tanh_layer", c.problem.eps, c.problem.alpha, c.problem.b, c.problem.exact)
    ma = W.structured_mesh(c.N)
    h = gpu_setup(ma, c.k, method, prob, tol=1e-12, gmres_m=50)
    run = oracle_run(ma, c.k, method, prob)
    xo = oracle_direct(run)
    T = basis_change(run, ma, c.k)
    for xg, tol in ((h.gmres_solve()[0], 1e-8), (h.dense_solve(), 1e-10)):
        np.testing.assert_allclose(x_to_oracle(T, _np(xg)), xo, rtol=0, atol=tol * np.abs(xo).max())
    xe = O.quad_points(run.mesh, c.k, O.ERROR)
    l2o, hmo = O.l2_error(run.mesh, c.k, xo, prob.u(np, xe[..., 0], xe[..., 1]))
    l2g, hmax = h.l2_error(xg, problem.exact_at_error_points(h, prob))
    assert abs(l2g - l2o) <= 1e-9 * l2o and abs(hmax - hmo) <= 1e-15
    h.close()


@pytest.mark.parametrize("k", [1, 2])
def test_solve_on_a_refined_polygonal_mesh(k):
    """uniformrefine (Sec. 2.1) of an L-shaped domain with Dirichlet and Neumann
    parts, three times (384 triangles), then the GPU solve: a P_k polynomial is
    reproduced, and the solution equals the oracle's direct solve on the same
    mesh as a function."""
    m = W.lshape_mesh()
    arrays = (m.nodes, m.elems, m.dirichlet, m.neumann)
    for _ in range(3):
        arrays = D.dg_mesh_refine(*arrays)
    ma = W.MeshArrays(*arrays)
    a, bb = {1: (1, 0), 2: (1, 1)}[k]
    prob = W.Problem("poly", 0.3, 0.7, (0.4, 0.3, -0.2, -0.6, 0.1, 0.5), W.polynomial(a, bb))
    h = gpu_setup(ma, k, 2, prob, tol=1e-12, gmres_m=50)
    x, _ = h.gmres_solve()
    l2, _ = h.l2_error(x, problem.exact_at_error_points(h, prob))
    assert l2 < 1e-9
    run = oracle_run(ma, k, 2, prob)
    xo = oracle_direct(run)
    T = basis_change(run, ma, k)
    np.testing.assert_allclose(x_to_oracle(T, _np(x)), xo, rtol=0, atol=1e-8 * np.abs(xo).max())
    h.close()


def test_captured_cycle_is_not_reused_across_degree_or_size():
    """The restart cycle captured as a CUDA graph bakes in the element count and
    the degree.  A P1 mesh and a P2 mesh with the same number of unknowns (384),
    solved in turn on one handle into the same output buffer, give the results
    of fresh handles."""
    m8 = W.structured_mesh(8)                                              # 128 triangles, P1
    m44, _ = W.concat_meshes([W.structured_mesh(4), W.structured_mesh(4)])   # 64 triangles, P2
    cases = [(W.sine_8x8(), m8), (W.boundary_layer_p2(method=2, N=4), m44)]
    h = D.DG(0)
    x = torch.empty(384, dtype=torch.float64, device="cuda")
    got = []
    for c, m in cases + cases:
        problem.setup(h, c, mesh=m, tol=1e-11, gmres_m=20)
        assert h.info().dofs == 384
        h.gmres_solve(x=x)
        got.append(_np(x).copy())
    h.close()
    for i, (c, m) in enumerate(cases):
        hf = D.DG(0)
        problem.setup(hf, c, mesh=m, tol=1e-11, gmres_m=20)
        xf, _ = hf.gmres_solve()
        xf = _np(xf)
        for g in (got[i], got[i + 2]):
            assert np.abs(g - xf).max() <= 1e-12 * np.abs(xf).max()
        hf.close()


@pytest.mark.parametrize("method", [1, 2])
def test_gmres_matches_oracle(method):
    cfg = W.boundary_layer_p2(method=method, N=12)
    ma = W.structured_mesh(cfg.N)
    h = gpu_setup(ma, cfg.k, cfg.method, cfg.problem, tol=1e-12, gmres_m=20)
    xg, info = h.gmres_solve()
    assert info.status == D.DG_OK and info.relres <= 1e-12
    run = oracle_run(ma, cfg.k, cfg.method, cfg.problem)
    T = basis_change(run, ma, cfg.k)
    assert rel_residual_oracle(run, T, _np(xg)) <= 1e-10
    xo = oracle_direct(run)
    assert np.abs(x_to_oracle(T, _np(xg)) - xo).max() <= 1e-8 * np.abs(xo).max()
    h.close()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_polynomial_reproduction_gpu(k):
    """u in P_k with exact data is reproduced by the GPU assembly + GMRES solve
    (independent of the oracle: the method's consistency)."""
    prob = _poly_problem(k)
    ma = W.perturbed_mesh(4, seed=7, neumann_sides=prob.neumann_sides)
    for method in (1, 2, 3):
        h = gpu_setup(ma, k, method, prob, tol=1e-13, gmres_m=30)
        xg, info = h.gmres_solve()
        l2, _ = h.l2_error(xg, problem.exact_at_error_points(h, prob))
        assert l2 < 1e-10, (method, l2, info.relres)
        h.close()


def test_eval_matches_oracle():
    prob = _bumpy_problem()
    ma = W.perturbed_mesh(3, seed=4, neumann_sides=prob.neumann_sides)
    k = 2
    h = gpu_setup(ma, k, 2, prob)
    run = oracle_run(ma, k, 2, prob)
    T = basis_change(run, ma, k)
    xg = np.random.default_rng(3).standard_normal(ma.ne * 6)
    rs = np.array([[0.1, 0.2], [0.5, 0.25], [0.3, 0.6]])
    ug = _np(h.eval(torch.tensor(xg, device="cuda"), rs))
    v = ma.nodes[ma.elems]
    xy = v[:, None, 0] + rs[None, :, 0, None] * (v[:, None, 1] - v[:, None, 0]) + rs[None, :, 1, None] * (v[:, None, 2] - v[:, None, 0])
    uo = O.evaluate(run.mesh, k, x_to_oracle(T, xg), np.repeat(np.arange(ma.ne), 3), xy.reshape(-1, 2))
    np.testing.assert_allclose(ug.reshape(-1), uo, rtol=0, atol=1e-12 * np.abs(uo).max())
    h.close()


def test_nonfinite_data_reported():
    cfg = W.boundary_layer_p2(N=4)
    ma = W.structured_mesh(cfg.N)
    h = D.DG(0)
    problem.setup(h, cfg, mesh=ma, assemble=False)
    f, gD, gN = problem.problem_data(h, cfg.problem)
    f[0, 0] = float("nan")
    p = cfg.problem
    h.assemble(p.eps, p.alpha, p.b, f, gD, gN)
    with pytest.raises(D.DGError) as e:
        h.gmres_solve()
    assert e.value.status == D.DG_ERR_NONFINITE
    h.close()


# ----------------------------------------------------------------------------
# mixed-precision refinement
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("inner", ["f32", "bf16"])
def test_mixed_refinement_reaches_f64_tolerance(inner):
    """bf16/f32 inner solves with f64 refinement reach rel-res 1e-10, measured
    by the oracle's own f64 operator (reading A-12)."""
    cfg = W.gaussian_bump_p3(N=12)
    ma = W.structured_mesh(cfg.N, cfg.problem.neumann_sides)
    store = D.DG_STORE_F64 | (D.DG_STORE_F32 if inner == "f32" else D.DG_STORE_BF16)
    h = gpu_setup(ma, cfg.k, cfg.method, cfg.problem, store=store, tol=1e-10)
    dt = D.DG_F32 if inner == "f32" else D.DG_BF16
    xg, info = h.mixed_solve(dt, inner_m=30, inner_tol=1e-4 if inner == "f32" else 1e-2, max_outer=40)
    assert info.status == D.DG_OK and info.relres <= 1e-10 and info.outer >= 1
    run = oracle_run(ma, cfg.k, cfg.method, cfg.problem)
    T = basis_change(run, ma, cfg.k)
    assert rel_residual_oracle(run, T, _np(xg)) <= 1e-10 * 1.5
    # same solution as the f64 GMRES path, as functions
    x64, _ = h.gmres_solve()
    xo = x_to_oracle(T, _np(x64))
    assert np.abs(x_to_oracle(T, _np(xg)) - xo).max() <= 1e-7 * np.abs(xo).max()
    h.close()


@pytest.mark.parametrize("inner", ["f32", "bf16"])
def test_gmres_refinement_reaches_f64_tolerance(inner):
    """Outer f64 FGMRES with the low-precision solve as preconditioner reaches
    rel-res 1e-10, measured by the oracle's own f64 operator (reading A-12)."""
    cfg = W.gaussian_bump_p3(N=12)
    ma = W.structured_mesh(cfg.N, cfg.problem.neumann_sides)
    store = D.DG_STORE_F64 | (D.DG_STORE_F32 if inner == "f32" else D.DG_STORE_BF16)
    h = gpu_setup(ma, cfg.k, cfg.method, cfg.problem, store=store, tol=1e-10)
    dt = D.DG_F32 if inner == "f32" else D.DG_BF16
    xg, info = h.gmres_ir_solve(dt, inner_m=30, inner_tol=1e-4 if inner == "f32" else 1e-2, max_outer=100)
    assert info.status == D.DG_OK and info.relres <= 1e-10 and info.outer >= 1
    run = oracle_run(ma, cfg.k, cfg.method, cfg.problem)
    T = basis_change(run, ma, cfg.k)
    assert rel_residual_oracle(run, T, _np(xg)) <= 1e-10 * 1.5
    h.close()


def test_gmres_refinement_converges_where_bf16_refinement_stalls():
    """The 256x256 boundary-layer workload at eps = 1e-6 (P2, SIPG): plain
    refinement around bf16 inner solves stalls (cond(A) u_bf16 > 1); the f64
    FGMRES outer loop around the same inner solves reaches 1e-10.  The final
    residual is re-measured here with the f64 apply."""
    cfg = W.boundary_layer_p2(method=2, N=256)
    ma = W.structured_mesh(cfg.N)
    h = gpu_setup(ma, cfg.k, cfg.method, cfg.problem, store=D.DG_STORE_F64 | D.DG_STORE_BF16, tol=1e-10,
                  max_it=4000)
    _, plain = h.mixed_solve(D.DG_BF16, inner_m=50, inner_tol=1e-2, max_outer=10, raise_on_nonconv=False)
    assert plain.status == D.DG_NOT_CONVERGED and plain.relres > 1e-3
    h.set_params(max_it=20000)
    xg, info = h.gmres_ir_solve(D.DG_BF16, inner_m=50, inner_tol=1e-2, max_outer=200)
    assert info.status == D.DG_OK and info.relres <= 1e-10
    F = h.rhs()
    rr = (torch.linalg.norm(F - h.apply(xg)) / torch.linalg.norm(F)).item()
    assert rr <= 1.5e-10
    h.close()


@pytest.mark.parametrize("solver", ["f64", "batch"])
def test_gmres_lucky_breakdown_on_block_diagonal_operator(solver):
    """eps = 0, b = 0: the operator is alpha times the block-diagonal mass
    matrix, block Jacobi inverts it exactly, so GMRES stops after one Arnoldi
    step through the breakdown path (the orthogonalised vector vanishes) with
    x = A^-1 F, the L2 projection of f / alpha."""
    prob = W.Problem("react", 0.0, 2.0, (0,) * 6, W.sinsin)
    ma = W.perturbed_mesh(6, seed=4)
    h = gpu_setup(ma, 2, 2, prob, tol=1e-12)
    h.precond_setup()
    xb = h.precond_apply(h.rhs(), D.DG_F64)
    if solver == "f64":
        x, info = h.gmres_solve()
        its, st = info.iterations, info.status
    else:
        h.batch_setup(np.array([0, ma.ne], np.int32), np.array([[0.0, 2.0, 0, 0, 0, 0, 0, 0]]))
        h.assemble(0.0, 2.0, (0,) * 6, *problem.problem_data(h, prob))
        h.precond_setup()
        x, its_a, rr, st_a = h.batch_solve(D.DG_F64)
        its, st = int(its_a[0]), int(st_a[0])
    assert st == D.DG_OK and its == 1
    np.testing.assert_allclose(_np(x), _np(xb), rtol=1e-12, atol=1e-14 * np.abs(_np(xb)).max())
    h.close()


# ----------------------------------------------------------------------------
# one-layer-overlap Schwarz preconditioner
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("k", [1, 2, 3])
def test_schwarz_apply_is_the_patch_solve(k):
    """z = M^-1 r equals, element by element, the patch solve of the oracle's
    definition (oracle/mlp.py patch_correction on the GPU's own blocks)."""
    from oracle import mlp as M
    prob = _bumpy_problem()
    ma = W.perturbed_mesh(5, seed=7, neumann_sides=prob.neumann_sides)
    h = gpu_setup(ma, k, 2, prob, store=D.DG_STORE_F64 | D.DG_STORE_F32)
    h.set_params(precond=D.DG_PRECOND_SCHWARZ)
    h.precond_setup(D.DG_PRECOND_SCHWARZ)
    A, nbr = h.blocks()
    A, nbr = _np(A), _np(nbr).astype(np.int64)
    nb = O.nbasis(k)
    r = np.random.default_rng(k).standard_normal(ma.ne * nb)
    z = _np(h.precond_apply(torch.tensor(r, device="cuda"), D.DG_F64))
    w = M.patch_correction(A, nbr, r, nb)
    assert np.abs(z - w).max() <= 1e-10 * np.abs(w).max()
    z32 = _np(h.precond_apply(torch.tensor(r, dtype=torch.float32, device="cuda"), D.DG_F32))
    assert np.abs(z32 - w).max() <= 1e-4 * np.abs(w).max()
    h.close()


def test_schwarz_gmres_reaches_tolerance_in_fewer_steps():
    """GMRES(50) with the Schwarz preconditioner on the boundary-layer workload
    (32x32, P2, NIPG): relres <= 1e-10 measured by the oracle's operator, in
    fewer Arnoldi steps than with block Jacobi; mixed refinement around f32
    Schwarz-preconditioned inner solves also reaches 1e-10."""
    cfg = W.boundary_layer_p2(method=1, N=32)
    ma = W.structured_mesh(cfg.N)
    h = gpu_setup(ma, cfg.k, cfg.method, cfg.problem, store=D.DG_STORE_F64 | D.DG_STORE_F32, tol=1e-10,
                  gmres_m=50)
    h.set_params(precond=D.DG_PRECOND_BLOCK_JACOBI)
    _, ib = h.gmres_solve()
    h.set_params(precond=D.DG_PRECOND_SCHWARZ)
    xs, iS = h.gmres_solve()
    assert iS.status == D.DG_OK and iS.iterations < ib.iterations
    run = oracle_run(ma, cfg.k, cfg.method, cfg.problem)
    T = basis_change(run, ma, cfg.k)
    assert rel_residual_oracle(run, T, _np(xs)) <= 1e-10 * 1.5
    xm, im = h.mixed_solve(D.DG_F32, inner_m=30, inner_tol=1e-3, max_outer=30)
    assert im.status == D.DG_OK and rel_residual_oracle(run, T, _np(xm)) <= 1e-10 * 1.5
    print(f"Arnoldi steps: block Jacobi {ib.iterations}, Schwarz {iS.iterations}")
    h.close()


@pytest.mark.parametrize("N,k", [(10, 2), (13, 3)])
def test_blocked_dense_lu_matches_oracle(N, k):
    """The blocked LU of the dense solve equals the oracle's direct solve as a
    function, and an all-zero operator is reported as singular.  1200 and 3380
    unknowns: panels of 16 (8, then 16) columns, as wide as the shared-memory
    panel allows for the rows left, the last one ragged; the 1200-unknown
    operator takes 490 row swaps under partial pivoting (LAPACK's getrf on
    the same matrix), so the pivoting path is exercised."""
    prob = W.Problem("gauss", 0.05, 0.4, (0.5, 0.0, -1.0, -0.5, 1.0, 0.0), W.gaussian_bump,
                     neumann_sides=("right", "top"))
    ma = W.perturbed_mesh(N, seed=3, neumann_sides=prob.neumann_sides)
    h = gpu_setup(ma, k, 1, prob)
    n = h.info().dofs
    assert n % 32 != 0
    xg = h.dense_solve()
    run = oracle_run(ma, k, 1, prob)
    xo = oracle_direct(run)
    T = basis_change(run, ma, k)
    assert np.abs(x_to_oracle(T, _np(xg)) - xo).max() <= 1e-10 * np.abs(xo).max()
    h.close()
    hz = gpu_setup(W.structured_mesh(3), 1, 2, W.Problem("z", 0.0, 0.0, (0,) * 6, W.sinsin))
    with pytest.raises(D.DGError) as e:
        hz.dense_solve()
    assert e.value.status == D.DG_ERR_SINGULAR_BLOCK
    hz.close()


@pytest.mark.parametrize("N,k", [(8, 1), (10, 2)])
def test_dense_solve_refined_f32_factors_and_f64_factors_agree(N, k, monkeypatch):
    """The dense solve's two paths: f32 factors with f64 refinement (the
    default) and f64 factors (DG_DENSE_F64=1 at dg_create) both equal the
    oracle's direct solve, their true residuals are at f64 rounding level, and
    F may be the output vector itself."""
    prob = W.Problem("gauss", 0.05, 0.4, (0.5, 0.0, -1.0, -0.5, 1.0, 0.0), W.gaussian_bump,
                     neumann_sides=("right", "top"))
    ma = W.perturbed_mesh(N, seed=5, neumann_sides=prob.neumann_sides)
    run = oracle_run(ma, k, 2, prob)
    xo = oracle_direct(run)
    T = basis_change(run, ma, k)
    xs = []
    for f64 in (False, True):
        if f64:
            monkeypatch.setenv("DG_DENSE_F64", "1")
        h = gpu_setup(ma, k, 2, prob)
        monkeypatch.delenv("DG_DENSE_F64", raising=False)
        xg = h.dense_solve()
        F = h.rhs()
        rr = (torch.linalg.norm(F - h.apply(xg)) / torch.linalg.norm(F)).item()
        assert rr <= 1e-13, (f64, rr)
        assert np.abs(x_to_oracle(T, _np(xg)) - xo).max() <= 1e-10 * np.abs(xo).max()
        xa = F.clone()
        h.check(D.dg_dense_solve(h.h, xa, xa))   # F and x the same vector
        assert torch.equal(xa, xg)
        xs.append(_np(xg))
        h.close()
    assert np.abs(xs[0] - xs[1]).max() <= 1e-11 * np.abs(xs[1]).max()
