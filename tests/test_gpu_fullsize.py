"""GPU parity at the launch shapes the full-size workloads take.

The small parity tests run every kernel in its small-grid shape.  These cases
reach the shapes the benchmark's workloads use:
  * the operator apply with 256-thread blocks (more element warps than
    32 per SM can hold), on a 300x300 split P1 mesh and on the 512x512 P3
    operator the benchmark times;
  * the 256x256 P2 boundary-layer solves of the benchmark step (f64 GMRES and
    the f32-refined solve), measured with the oracle's own FP64 operator
    (reading A-12 of the paper's "match" for iterative solves);
  * batched solves whose instances span several work items of the segmented
    reductions (per-instance arrival counters and multi-item partial sums).
Tolerances are those of the small parity tests: f64 applies entry by entry at
1e-11 of the largest entry through the basis change, iterative solutions at an
oracle-measured relative residual of 1.5e-10 (the GPU's own stop test is
1e-10 with its own operator), batch against single-instance solves at 1e-8.
"""
import numpy as np
import pytest

import oracle as O
from paper_1502_02941_gb300 import dg as D
from paper_1502_02941_gb300 import problem
from paper_1502_02941_gb300 import workloads as W
from gpu_helpers import basis_change, gpu_setup, oracle_run, rel_residual_oracle, x_to_oracle
from helpers import oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def _nsm():
    return torch.cuda.get_device_properties(0).multi_processor_count


def _ref_apply(A, nbr, x, ne, nb):
    X = x.reshape(ne, nb)
    y = np.einsum("kij,kj->ki", A[:, 0], X)
    for f in range(3):
        L = nbr[:, f]
        ok = L >= 0
        y[ok] += np.einsum("kij,kj->ki", A[ok, 1 + f], X[L[ok]])
    return y.reshape(-1)


def _apply_against_oracle(h, ma, k, method, prob, seed):
    run = oracle_run(ma, k, method, prob, split=False)
    T = basis_change(run, ma, k)
    nb = O.nbasis(k)
    xg = np.random.default_rng(seed).standard_normal(ma.ne * nb)
    yg = _np(h.apply(torch.tensor(xg, device="cuda"), D.DG_F64))
    yo = O.apply(run.mesh, run.system.A_diag, run.system.A_off, x_to_oracle(T, xg))
    yo_g = np.einsum("kmi,km->ki", T, yo.reshape(ma.ne, nb)).reshape(-1)
    err = np.abs(yg - yo_g).max() / np.abs(yo_g).max()
    assert err <= 1e-11, err
    return xg


def _low_precision_applies(h, ma, nb, xg):
    """f32 / bf16 applies equal the same stored blocks evaluated in f64, up to
    f32 accumulation."""
    xt = torch.tensor(xg, device="cuda", dtype=torch.float32)
    x64 = _np(xt.double())
    for dt in (D.DG_F32, D.DG_BF16):
        Alo, nbr = h.blocks(dt)
        Alo, nbr = _np(Alo.double()), _np(nbr)
        ylo = _np(h.apply(xt, dt).double())
        yref = _ref_apply(Alo, nbr, x64, ma.ne, nb)
        err = np.abs(ylo - yref).max() / np.abs(yref).max()
        assert err <= 2e-6, (dt, err)
        del Alo


def test_apply_parity_with_256_thread_blocks_p1():
    """300x300 split squares (180,000 triangles, perturbed), P1: more element
    warps than 32 per SM, so the apply runs 256-thread blocks."""
    prob = W.Problem("gauss", 0.05, 0.4, (0.5, 0.0, -1.0, -0.5, 1.0, 0.0), W.gaussian_bump,
                     neumann_sides=("right", "top"))
    ma = W.perturbed_mesh(300, seed=5, neumann_sides=prob.neumann_sides)
    assert (ma.ne + 31) // 32 > 32 * _nsm()
    h = gpu_setup(ma, 1, 1, prob, store=D.DG_STORE_F64 | D.DG_STORE_F32 | D.DG_STORE_BF16)
    xg = _apply_against_oracle(h, ma, 1, 1, prob, seed=1)
    _low_precision_applies(h, ma, 3, xg)
    h.close()


def test_apply_parity_on_the_512x512_p3_operator():
    """The 512x512 P3 Gaussian-bump operator (524,288 triangles, 5.24 M
    unknowns) in the configuration the benchmark times: f64 apply against the
    oracle element by element, f32 / bf16 against their stored blocks."""
    cfg = W.gaussian_bump_p3(N=512)
    ma = W.structured_mesh(cfg.N, cfg.problem.neumann_sides)
    h = D.DG(0)
    problem.setup(h, cfg, store=D.DG_STORE_F64 | D.DG_STORE_F32 | D.DG_STORE_BF16, mesh=ma)
    assert (ma.ne + 31) // 32 > 32 * _nsm()
    xg = _apply_against_oracle(h, ma, cfg.k, cfg.method, cfg.problem, seed=2)
    _low_precision_applies(h, ma, 10, xg)
    h.close()


@pytest.mark.parametrize("method", [1, 2])
def test_full_size_solves_reach_tolerance_with_the_oracle_operator(method):
    """The benchmark step's 256x256 P2 boundary-layer solve (eps = 1e-6,
    b = (1,0), alpha = 1): f64 GMRES(50) + block Jacobi, and the f32-refined
    solve (f32 GMRES(32) inner solves to 1e-3, f64 residual correction), both
    to 1e-10 by the library's stop test; the residual of each solution with the
    oracle's own f64 operator is at most 1.5e-10."""
    cfg = W.boundary_layer_p2(method=method, N=256)
    ma = W.structured_mesh(cfg.N)
    h = gpu_setup(ma, cfg.k, cfg.method, cfg.problem, store=D.DG_STORE_F64 | D.DG_STORE_F32, tol=1e-10,
                  gmres_m=50, max_it=20000)
    h.precond_setup()
    x64, i64 = h.gmres_solve()
    assert i64.status == D.DG_OK and i64.relres <= 1e-10
    x32, i32 = h.mixed_solve(D.DG_F32, inner_m=32, inner_tol=1e-3, max_outer=60)
    assert i32.status == D.DG_OK and i32.relres <= 1e-10
    run = oracle_run(ma, cfg.k, cfg.method, cfg.problem, split=False)
    T = basis_change(run, ma, cfg.k)
    r64 = rel_residual_oracle(run, T, _np(x64))
    r32 = rel_residual_oracle(run, T, _np(x32))
    print(f"oracle-measured relres: f64 GMRES {r64:.3e} ({i64.iterations} steps), "
          f"f32-refined {r32:.3e} ({i32.iterations} inner steps)")
    assert r64 <= 1.5e-10 and r32 <= 1.5e-10
    h.close()


def _check_batch_against_oracle_and_single(cfgs, starts, xb, store, solve_single):
    nb = O.nbasis(cfgs[0].k)
    for i, c in enumerate(cfgs):
        a, b = starts[i] * nb, starts[i + 1] * nb
        mi = W.structured_mesh(c.N)
        run = oracle_system(mi, c.k, c.method, c.problem)
        T = basis_change(run, mi, c.k)
        rr = rel_residual_oracle(run, T, xb[a:b])
        assert rr <= 1e-10, (i, rr)
        hs = D.DG(0)
        problem.setup(hs, c, mesh=mi, tol=1e-11, gmres_m=20, store=store)
        xs = _np(solve_single(hs))
        assert np.abs(xs - xb[a:b]).max() <= 1e-8 * np.abs(xs).max(), i
        hs.close()


@pytest.mark.parametrize("inner", ["f64", "f32", "bf16_gmres_ir"])
def test_batch_instances_spanning_several_work_items(inner):
    """Work items of 256 unknowns: every P2 instance (N in [8, 12], 768 to 1728
    unknowns) spans 3 to 7 items, so each reduction is a multi-item segmented
    sum closed by the instance's last item to arrive."""
    cfgs, ma, starts, coeffs = W.batch("batched", 4, k=2, N_range=(8, 12))
    nb = 6
    assert all((starts[i + 1] - starts[i]) * nb > 2 * 256 for i in range(len(cfgs)))
    h = D.DG(0)
    store = D.DG_STORE_F64 | {"f64": 0, "f32": D.DG_STORE_F32, "bf16_gmres_ir": D.DG_STORE_BF16}[inner]
    problem.setup_batch(h, cfgs, ma, starts, coeffs, store=store, tol=1e-11, gmres_m=20)
    h.precond_setup()
    h.check(D.dg_batch_set_tile(h.h, 256))
    if inner == "f64":
        x, its, rr, st = h.batch_solve(D.DG_F64)
        single = lambda hs: hs.gmres_solve()[0]
    elif inner == "f32":
        x, its, rr, st = h.batch_solve(D.DG_F32, inner_m=20, inner_tol=1e-5, max_outer=30)
        single = lambda hs: hs.gmres_solve()[0]
    else:
        x, its, rr, st = h.batch_gmres_ir_solve(D.DG_BF16, inner_m=16, inner_tol=1e-2, max_outer=300)
        single = lambda hs: hs.gmres_ir_solve(D.DG_BF16, inner_m=16, inner_tol=1e-2, max_outer=300)[0]
    assert (st == 0).all() and (rr <= 1e-11).all() and (its > 0).all()
    _check_batch_against_oracle_and_single(cfgs, starts, _np(x), store, single)
    h.close()


def test_batch_large_instances_at_the_default_tile():
    """Two P2 instances with N = 40 and 48 (19,200 and 27,648 unknowns) at the
    default work item of 4096 unknowns (5 and 7 items each), f32 GMRES-based
    refinement with the Schwarz preconditioner, as the benchmark runs it."""
    cfgs = [W.random_instance("batched", i, N_fixed=N, k_fixed=2) for i, N in ((0, 40), (1, 48))]
    ma, starts = W.concat_meshes([W.structured_mesh(c.N) for c in cfgs])
    coeffs = np.array([[c.problem.eps, c.problem.alpha, *c.problem.b] for c in cfgs])
    h = D.DG(0)
    store = D.DG_STORE_F64 | D.DG_STORE_F32
    problem.setup_batch(h, cfgs, ma, starts, coeffs, store=store, tol=1e-11, gmres_m=50,
                        precond=D.DG_PRECOND_SCHWARZ, max_it=20000)
    h.check(D.dg_batch_set_tile(h.h, 0))
    x, its, rr, st = h.batch_gmres_ir_solve(D.DG_F32, inner_m=32, inner_tol=1e-3, max_outer=1000)
    assert (st == 0).all() and (rr <= 1e-11).all()
    xb = _np(x)
    for i, c in enumerate(cfgs):
        a, b = starts[i] * 6, starts[i + 1] * 6
        assert b - a > 4 * 4096
        mi = W.structured_mesh(c.N)
        run = oracle_system(mi, c.k, c.method, c.problem)
        T = basis_change(run, mi, c.k)
        assert rel_residual_oracle(run, T, xb[a:b]) <= 1e-10
    h.close()
