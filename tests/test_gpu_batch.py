"""Batched solves of independent instances (per-instance reductions and
convergence) against single-instance solves and the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1502_02941_gb300 import dg as D
from paper_1502_02941_gb300 import problem
from paper_1502_02941_gb300 import workloads as W
from gpu_helpers import basis_change, rel_residual_oracle
from helpers import oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_batch_matches_single_instance_solves(k, inner):
    cfgs, ma, starts, coeffs = W.batch("batched", 5, k=k, N_range=(3, 7))
    h = D.DG(0)
    store = D.DG_STORE_F64 | (D.DG_STORE_F32 if inner == "f32" else 0)
    problem.setup_batch(h, cfgs, ma, starts, coeffs, store=store, tol=1e-11, gmres_m=20)
    h.precond_setup()
    dt = D.DG_F64 if inner == "f64" else D.DG_F32
    x, its, rr, st = h.batch_solve(dt, inner_m=20, inner_tol=1e-5, max_outer=30)
    assert (st == 0).all() and (rr <= 1e-11).all() and (its > 0).all()
    xb = _np(x)
    nb = O.nbasis(k)
    for i, c in enumerate(cfgs):
        a, b = starts[i] * nb, starts[i + 1] * nb
        mi = W.structured_mesh(c.N)
        # oracle: residual of this instance's GPU solution with the oracle operator
        run = oracle_system(mi, c.k, c.method, c.problem)
        T = basis_change(run, mi, c.k)
        assert rel_residual_oracle(run, T, xb[a:b]) <= 1e-10
        # single-instance GPU solve of the same instance
        hs = D.DG(0)
        problem.setup(hs, c, mesh=mi, tol=1e-11, gmres_m=20)
        xs, _ = hs.gmres_solve()
        xs = _np(xs)
        assert np.abs(xs - xb[a:b]).max() <= 1e-8 * np.abs(xs).max()
        hs.close()
    h.close()


def test_batch_autotune_and_rejects_touching_instances():
    cfgs, ma, starts, coeffs = W.batch("batched", 4, k=1, N_range=(3, 5))
    h = D.DG(0)
    problem.setup_batch(h, cfgs, ma, starts, coeffs)
    tile = h.batch_autotune()
    assert tile in (2048, 4096, 8192, 16384, 32768)
    x, its, rr, st = h.batch_solve(D.DG_F64, raise_on_nonconv=False)
    assert (st == 0).all()
    # one mesh declared as two instances: they share edges
    m = W.structured_mesh(4)
    h.mesh_upload(m.nodes, m.elems, m.dirichlet, m.neumann)
    with pytest.raises(D.DGError) as e:
        h.batch_setup(np.array([0, 10, m.ne], np.int32), np.zeros((2, 8)))
    assert e.value.status == D.DG_ERR_MESH
    h.close()


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_batch_with_schwarz_matches_oracle(inner):
    """Batched solve with the Schwarz preconditioner: every instance reaches
    1e-10 measured by the oracle's operator, in no more Arnoldi steps than with
    block Jacobi."""
    cfgs, ma, starts, coeffs = W.batch("batched", 5, k=2, N_range=(4, 8))
    h = D.DG(0)
    store = D.DG_STORE_F64 | (D.DG_STORE_F32 if inner == "f32" else 0)
    problem.setup_batch(h, cfgs, ma, starts, coeffs, store=store, tol=1e-11, gmres_m=20)
    dt = D.DG_F64 if inner == "f64" else D.DG_F32
    h.set_params(precond=D.DG_PRECOND_BLOCK_JACOBI)
    _, its_bj, _, _ = h.batch_solve(dt, inner_m=20, inner_tol=1e-5, max_outer=30)
    h.set_params(precond=D.DG_PRECOND_SCHWARZ)
    x, its, rr, st = h.batch_solve(dt, inner_m=20, inner_tol=1e-5, max_outer=30)
    assert (st == 0).all() and (rr <= 1e-11).all()
    assert its.sum() <= its_bj.sum()
    xb = _np(x)
    nb = O.nbasis(2)
    for i, c in enumerate(cfgs):
        a, b = starts[i] * nb, starts[i + 1] * nb
        mi = W.structured_mesh(c.N)
        run = oracle_system(mi, c.k, c.method, c.problem)
        T = basis_change(run, mi, c.k)
        assert rel_residual_oracle(run, T, xb[a:b]) <= 1e-10
    h.close()


@pytest.mark.parametrize("inner,pc", [("f32", "bj"), ("bf16", "bj"), ("f32", "schwarz")])
def test_batch_gmres_refinement_matches_oracle(inner, pc):
    """Batched GMRES-based refinement (f64 flexible GMRES per instance around the
    batched low-precision inner solve): every instance reaches 1e-11 in its own
    f64 residual and 1e-10 measured by the oracle's operator, and agrees with
    the single-instance GMRES-based refinement of the same instance."""
    cfgs, ma, starts, coeffs = W.batch("batched", 5, k=2, N_range=(4, 8))
    h = D.DG(0)
    store = D.DG_STORE_F64 | (D.DG_STORE_F32 if inner == "f32" else D.DG_STORE_BF16)
    prec = D.DG_PRECOND_SCHWARZ if pc == "schwarz" else D.DG_PRECOND_BLOCK_JACOBI
    problem.setup_batch(h, cfgs, ma, starts, coeffs, store=store, tol=1e-11, gmres_m=20, precond=prec)
    dt = D.DG_F32 if inner == "f32" else D.DG_BF16
    itol = 1e-3 if inner == "f32" else 1e-2
    x, its, rr, st = h.batch_gmres_ir_solve(dt, inner_m=16, inner_tol=itol, max_outer=200)
    assert (st == 0).all() and (rr <= 1e-11).all() and (its > 0).all()
    xb = _np(x)
    nb = O.nbasis(2)
    for i, c in enumerate(cfgs):
        a, b = starts[i] * nb, starts[i + 1] * nb
        mi = W.structured_mesh(c.N)
        run = oracle_system(mi, c.k, c.method, c.problem)
        T = basis_change(run, mi, c.k)
        assert rel_residual_oracle(run, T, xb[a:b]) <= 1e-10
        hs = D.DG(0)
        problem.setup(hs, c, mesh=mi, tol=1e-11, gmres_m=20, store=store, precond=prec)
        xs, info = hs.gmres_ir_solve(dt, inner_m=16, inner_tol=itol, max_outer=200)
        xs = _np(xs)
        assert np.abs(xs - xb[a:b]).max() <= 1e-8 * np.abs(xs).max()
        hs.close()
    # the learned correction is not an inner preconditioner; f64 is not an inner precision
    h.set_params(precond=D.DG_PRECOND_MLP)
    with pytest.raises(D.DGError) as e:
        h.batch_gmres_ir_solve(dt)
    assert e.value.status == D.DG_ERR_INVALID_ARG
    h.set_params(precond=prec)
    with pytest.raises(D.DGError) as e:
        h.batch_gmres_ir_solve(D.DG_F64)
    assert e.value.status == D.DG_ERR_INVALID_ARG
    h.close()


def test_batch_rejects_mixed_degrees():
    cfgs, ma, starts, coeffs = W.batch("batched", 6)
    assert len({c.k for c in cfgs}) == 2
    h = D.DG(0)
    with pytest.raises(ValueError):
        problem.setup_batch(h, cfgs, ma, starts, coeffs)
    h.close()


@pytest.mark.parametrize("solver", ["gmres_ir", "refine"])
def test_group_solve_of_a_mixed_degree_batch(solver):
    """Instances of the batched workload with both drawn degrees: one batch per
    degree, solved in one group call whose batches run concurrently on their
    own streams.  Every instance meets 1e-10 with the oracle's operator, and
    each batch's result equals its own single-batch solve."""
    groups = W.batch_by_degree("batched", 8, N_range=(4, 9))
    assert sorted(groups) == [1, 2]
    dgs, setups = [], []
    for k, (cfgs, ma, starts, coeffs) in groups.items():
        h = D.DG(0)
        problem.setup_batch(h, cfgs, ma, starts, coeffs, store=D.DG_STORE_F64 | D.DG_STORE_F32, tol=1e-11,
                            gmres_m=20, precond=D.DG_PRECOND_SCHWARZ)
        h.precond_setup(D.DG_PRECOND_SCHWARZ)
        dgs.append(h)
        setups.append((cfgs, starts))
    if solver == "gmres_ir":
        res = D.batch_group(dgs, "gmres_ir", D.DG_F32, inner_m=16, inner_tol=1e-3, max_outer=300)
    else:
        res = D.batch_group(dgs, "refine", D.DG_F32, inner_m=20, inner_tol=1e-5, max_outer=30)
    for h, (cfgs, starts), (x, its, rr, st) in zip(dgs, setups, res):
        assert (st == 0).all() and (rr <= 1e-11).all()
        if solver == "gmres_ir":
            xs, _, _, _ = h.batch_gmres_ir_solve(D.DG_F32, inner_m=16, inner_tol=1e-3, max_outer=300)
        else:
            xs, _, _, _ = h.batch_solve(D.DG_F32, inner_m=20, inner_tol=1e-5, max_outer=30)
        np.testing.assert_allclose(_np(x), _np(xs), rtol=0, atol=1e-12 * np.abs(_np(xs)).max())
        xb = _np(x)
        nb = O.nbasis(cfgs[0].k)
        for i, c in enumerate(cfgs):
            a, b = starts[i] * nb, starts[i + 1] * nb
            mi = W.structured_mesh(c.N)
            run = oracle_system(mi, c.k, c.method, c.problem)
            T = basis_change(run, mi, c.k)
            assert rel_residual_oracle(run, T, xb[a:b]) <= 1e-10
    # a handle twice is refused
    s = D.dg_batch_group_solve([dgs[0].h, dgs[0].h], D.DG_F32, 20, 1e-5, 30, None,
                               [res[0][0], res[0][0]])
    assert s == D.DG_ERR_INVALID_ARG
    for h in dgs:
        h.close()


def _pentagon():
    """Five triangles around a centre node (an odd element count), all
    boundary edges Dirichlet."""
    ang = np.pi / 2 + 2 * np.pi * np.arange(5) / 5
    nodes = np.vstack([[0.5, 0.5], np.column_stack([0.5 + 0.4 * np.cos(ang), 0.5 + 0.4 * np.sin(ang)])])
    elems = np.array([[0, 1 + i, 1 + (i + 1) % 5] for i in range(5)], np.int32)
    dirichlet = np.array([[1 + i, 1 + (i + 1) % 5] for i in range(5)], np.int32)
    return W.MeshArrays(nodes, elems, dirichlet, np.zeros((0, 2), np.int32))


@pytest.mark.parametrize("solver", ["refine", "gmres_ir"])
def test_batch_with_odd_unknown_offsets(solver):
    """P1 instances of 5, 20 and 5 triangles: the unknown offsets of the second
    and third instance are odd, so the f32 batched kernels take their scalar
    paths; each instance equals its single-instance solve."""
    p5 = _pentagon()
    p20 = W.MeshArrays(*D.dg_mesh_refine(p5.nodes, p5.elems, p5.dirichlet, p5.neumann))
    meshes = [p5, p20, p5]
    ma, starts = W.concat_meshes(meshes)
    assert (starts[1] * 3) % 2 == 1
    probs = [W.Problem("g", e, a, b, None, W.gaussians_source([(0.4, 0.6)], [0.15]))
             for e, a, b in ((0.05, 0.3, (0.6, 0, 0, -0.2, 0, 0)), (1e-3, 0.8, (0.1, 0, 0, 0.7, 0, 0)),
                             (0.2, 0.0, (-0.4, 0, 0, 0.1, 0, 0)))]
    cfgs = [W.Config(f"p{i}", 0, 1, 2, p) for i, p in enumerate(probs)]
    coeffs = np.array([[p.eps, p.alpha, *p.b] for p in probs])
    h = D.DG(0)
    store = D.DG_STORE_F64 | D.DG_STORE_F32
    problem.setup_batch(h, cfgs, ma, starts, coeffs, store=store, tol=1e-11, gmres_m=20)
    h.precond_setup()
    if solver == "refine":
        x, its, rr, st = h.batch_solve(D.DG_F32, inner_m=20, inner_tol=1e-5, max_outer=30)
    else:
        x, its, rr, st = h.batch_gmres_ir_solve(D.DG_F32, inner_m=16, inner_tol=1e-3, max_outer=300)
    assert (st == 0).all() and (rr <= 1e-11).all()
    xb = _np(x)
    for i, (c, mi) in enumerate(zip(cfgs, meshes)):
        a, b = starts[i] * 3, starts[i + 1] * 3
        hs = D.DG(0)
        problem.setup(hs, c, mesh=mi, tol=1e-12, gmres_m=20)
        xs = _np(hs.gmres_solve()[0])
        assert np.abs(xs - xb[a:b]).max() <= 1e-8 * np.abs(xs).max(), i
        hs.close()
    h.close()
