"""Learned preconditioner: GPU training/inference kernels against the FP64
oracle of the network (oracle/mlp.py), feature rows, and flexible GMRES."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_1502_02941_gb300 import dg as D
from paper_1502_02941_gb300 import problem
from paper_1502_02941_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def _handle(k=2, N=6):
    cfg = W.boundary_layer_p2(method=2, N=N)
    cfg.k = k
    h = D.DG(0)
    problem.setup(h, cfg, tol=1e-11, gmres_m=30)
    h.precond_setup()
    return h, cfg


@pytest.mark.parametrize("k", [1, 2])
def test_loss_and_gradient_match_oracle(k):
    """GPU loss/gradient (dg_mlp_loss_grad's default f32 GEMMs, bf16-rounded
    weights) vs the FP64 oracle backpropagation on the same bf16-rounded
    weights."""
    h, _ = _handle(k)
    nb = O.nbasis(k)
    rng = np.random.default_rng(k)
    theta = (rng.standard_normal(M.n_params(nb)) * 0.1).astype(np.float32)
    h.mlp_set_weights(theta)
    rows = 300
    X = rng.standard_normal((rows, M.din_of(nb))).astype(np.float32)
    T = rng.standard_normal((rows, nb)).astype(np.float32)
    grad = np.zeros(M.n_params(nb), np.float32)
    s, loss = D.dg_mlp_loss_grad(h.h, torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"), rows, grad)
    assert s == D.DG_OK
    lo, go = M.loss_and_grad(M.bf16_round_params(theta), X.astype(np.float64), T.astype(np.float64), nb)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    assert np.abs(grad - go).max() <= 2e-5 * np.abs(go).max()
    h.close()


def _oracle_loss_grad_bf16_gemms(theta, X, T, nb):
    """The oracle's backpropagation (oracle/mlp.py loss_and_grad) with the
    tensor-core path's roundings: every GEMM operand rounded to bf16 (the
    weights already are), accumulation, masks and bias sums unrounded."""
    W1, b1, W2, b2, W3, b3, W4, b4 = M.unpack(M.bf16_round_params(theta), nb)
    r = M.bf16_round
    a1 = r(X) @ W1.T + b1
    h1 = np.maximum(a1, 0)
    a2 = r(h1) @ W2.T + b2
    h2 = np.maximum(a2, 0)
    a3 = r(h2) @ W3.T + b3
    h3 = np.maximum(a3, 0)
    y = r(h3) @ W4.T + b4
    n = X.shape[0]
    d = (y - T) / n
    loss = 0.5 * ((y - T) ** 2).sum() / n
    gW4, gb4 = r(d).T @ r(h3), d.sum(0)
    d3 = (r(d) @ W4) * (a3 > 0)
    gW3, gb3 = r(d3).T @ r(h2), d3.sum(0)
    d2 = (r(d3) @ W3) * (a2 > 0)
    gW2, gb2 = r(d2).T @ r(h1), d2.sum(0)
    d1 = (r(d2) @ W2) * (a1 > 0)
    gW1, gb1 = r(d1).T @ r(X), d1.sum(0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4)] + [np.zeros(1)])
    return loss, g


@pytest.mark.parametrize("k,rows", [(1, 300), (2, 300), (2, 5000), (3, 300)])
def test_tensor_core_gradient_matches_oracle_with_bf16_operands(k, rows, monkeypatch):
    """The training GEMMs on the tensor cores (tcgen05, bf16 operands, f32
    accumulation; DG_MLP_GRAD_TC=1 routes dg_mlp_loss_grad through them, as
    dg_mlp_train always does) against the oracle's backpropagation with the
    same operand roundings.  300 rows leave ragged row tiles and K chunks;
    5000 rows split the weight gradients' K over many CTAs."""
    monkeypatch.setenv("DG_MLP_GRAD_TC", "1")
    h, _ = _handle(k)
    monkeypatch.delenv("DG_MLP_GRAD_TC")
    nb = O.nbasis(k)
    rng = np.random.default_rng(10 + k)
    theta = (rng.standard_normal(M.n_params(nb)) * 0.1).astype(np.float32)
    h.mlp_set_weights(theta)
    X = rng.standard_normal((rows, M.din_of(nb))).astype(np.float32)
    T = rng.standard_normal((rows, nb)).astype(np.float32)
    grad = np.zeros(M.n_params(nb), np.float32)
    s, loss = D.dg_mlp_loss_grad(h.h, torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"), rows, grad)
    assert s == D.DG_OK
    lo, go = _oracle_loss_grad_bf16_gemms(theta, X.astype(np.float64), T.astype(np.float64), nb)
    assert abs(loss - lo) <= 1e-4 * abs(lo)
    # (an intermediate can round to the neighbouring bf16 value when f32 and
    # f64 differ in its last bits: a few such entries, each a 2^-8 change of one
    # term of a long sum)
    assert np.abs(grad - go).max() <= 1e-3 * np.abs(go).max()
    # the f32 gradient of the same weights differs by about the bf16 rounding
    _, gf = M.loss_and_grad(M.bf16_round_params(theta), X.astype(np.float64), T.astype(np.float64), nb)
    assert np.abs(grad - gf).max() <= 5e-2 * np.abs(gf).max()
    h.close()


def _oracle_forward_bf16(theta, X, nb):
    """Oracle forward with the kernel's roundings: bf16 weights, inputs and
    hidden activations; f64 arithmetic otherwise."""
    W1, b1, W2, b2, W3, b3, W4, b4 = M.unpack(M.bf16_round_params(theta), nb)
    r = M.bf16_round
    h = r(np.maximum(r(X) @ W1.T + b1, 0))
    h = r(np.maximum(h @ W2.T + b2, 0))
    h = r(np.maximum(h @ W3.T + b3, 0))
    return h @ W4.T + b4


@pytest.mark.parametrize("k", [1, 2, 3])
def test_tensor_core_forward_matches_oracle(k):
    h, _ = _handle(k)
    nb = O.nbasis(k)
    rng = np.random.default_rng(10 + k)
    theta = (rng.standard_normal(M.n_params(nb)) * 0.15).astype(np.float32)
    h.mlp_set_weights(theta)
    rows = 517   # several 128-row tiles and a ragged tail
    X = rng.standard_normal((rows, M.din_of(nb))).astype(np.float32)
    Y = torch.zeros((rows, nb), dtype=torch.float32, device="cuda")
    assert D.dg_mlp_forward(h.h, torch.tensor(X, device="cuda"), rows, Y) == D.DG_OK
    yo = _oracle_forward_bf16(theta, X.astype(np.float64), nb)
    assert np.abs(_np(Y) - yo).max() <= 2e-2 * np.abs(yo).max()
    h.close()


def test_feature_rows_match_oracle():
    h, cfg = _handle(2, N=5)
    h.mlp_init(seed=3)
    nb = 6
    info = h.info()
    xk = torch.zeros(info.dofs, dtype=torch.float64, device="cuda")
    h.mlp_collect(xk)
    assert h.mlp_rows() == info.ne
    X = np.zeros((info.ne, M.din_of(nb)), np.float32)
    T = np.zeros((info.ne, nb), np.float32)
    assert D.dg_mlp_get_rows(h.h, X, T, info.ne) == D.DG_OK
    # oracle features from the same GPU residual r = F - A xk = F
    F = _np(h.rhs())
    A, nbr = h.blocks()
    A = _np(A)
    nbr = _np(nbr).astype(np.int64)
    p = cfg.problem
    geo_c = np.zeros((info.ne, 8))
    ma = W.structured_mesh(cfg.N)
    v = ma.nodes[ma.elems]
    cen = v.mean(1)
    J = np.stack([v[:, 1, 0] - v[:, 0, 0], v[:, 2, 0] - v[:, 0, 0], v[:, 1, 1] - v[:, 0, 1], v[:, 2, 1] - v[:, 0, 1]], 1)
    det = J[:, 0] * J[:, 3] - J[:, 1] * J[:, 2]
    geo_c[:, 4:8] = J / np.sqrt(det)[:, None]
    geo_c[:, 0] = p.eps
    geo_c[:, 1] = p.b[0] + p.b[1] * cen[:, 0] + p.b[2] * cen[:, 1]
    geo_c[:, 2] = p.b[3] + p.b[4] * cen[:, 0] + p.b[5] * cen[:, 1]
    geo_c[:, 3] = p.alpha
    Xo, so = M.features(F, nbr, nb, geo_c)
    np.testing.assert_allclose(X, Xo, rtol=2e-6, atol=2e-6)
    To = M.target(A, nbr, F, nb, so)
    np.testing.assert_allclose(T, To, rtol=1e-5, atol=1e-5 * np.abs(To).max())
    h.close()


def test_flexible_gmres_with_mlp_converges():
    """A randomly initialised network is a poor but valid preconditioner:
    flexible GMRES still reaches the tolerance, falling back to block Jacobi if
    it stalls; the residual is re-measured with the oracle's own f64 operator
    (reading A-12)."""
    from gpu_helpers import basis_change, oracle_run, rel_residual_oracle
    h, cfg = _handle(2, N=8)
    h.mlp_init(seed=1)
    h.set_params(precond=D.DG_PRECOND_MLP)
    x, info = h.gmres_solve()
    assert info.status == D.DG_OK and info.relres <= 1e-11
    ma = problem.mesh_for(cfg)
    run = oracle_run(ma, cfg.k, cfg.method, cfg.problem)
    T = basis_change(run, ma, cfg.k)
    assert rel_residual_oracle(run, T, _np(x)) <= 1e-10
    h.set_params(precond=D.DG_PRECOND_BLOCK_JACOBI)
    xb, ib = h.gmres_solve()
    assert np.abs(_np(x) - _np(xb)).max() <= 1e-8 * np.abs(_np(xb)).max()
    h.close()


def test_training_reduces_loss():
    h, cfg = _handle(2, N=12)
    h.mlp_init(seed=2)
    for its in (5, 15, 40):
        h.set_params(max_it=its)
        xk, _ = h.gmres_solve(raise_on_nonconv=False)
        h.mlp_collect(xk)
    loss = h.mlp_train(300, batch_rows=1024, lr=2e-3, seed=5)
    assert loss[-20:].mean() < 0.5 * loss[:5].mean()
    h.close()


def test_trained_network_fits_the_patch_correction_on_unseen_instances():
    """What training buys in the quantity it is trained on: on instances not
    seen in training, the trained network's preconditioner is at least twice as
    close (in the residual-space loss) to the one-layer-overlap Schwarz
    correction as block Jacobi alone (the untrained output y = 0); flexible
    GMRES with it still reaches the tolerance in f64 on every instance.  This
    is not a gain in Arnoldi steps or time: the test prints the measured step
    ratio, and the benchmark's learned section reports steps and time against
    block Jacobi and Schwarz."""
    from paper_1502_02941_gb300 import learned as L
    h = D.DG(0)
    L.make_batch(h, 16, 16, first=0, gmres_m=30)
    h.mlp_init(seed=4)
    L.collect(h, snapshots=(10, 40), basis_at=(20, 50), nvec=20)
    L.train(h, steps=2000, batch_rows=4096)
    th = h.mlp_get_weights()
    sigma = float(th[-1])
    he = D.DG(0)
    L.make_batch(he, 6, 16, first=5000, gmres_m=30)
    he.mlp_init(seed=0)
    L.collect(he, snapshots=(10, 40), basis_at=(20, 50), nvec=20)
    rows = he.mlp_rows()
    nb = 6
    X = torch.zeros((rows, M.din_of(nb)), dtype=torch.float32, device="cuda")
    T = torch.zeros((rows, nb), dtype=torch.float32, device="cuda")
    Xh = np.zeros((rows, M.din_of(nb)), np.float32)
    Th = np.zeros((rows, nb), np.float32)
    assert D.dg_mlp_get_rows(he.h, Xh, Th, rows) == D.DG_OK
    X.copy_(torch.from_numpy(Xh))
    T.copy_(torch.from_numpy(Th / sigma))
    he.mlp_set_weights(th)
    s, loss_trained = D.dg_mlp_loss_grad(he.h, X, T, rows)
    assert s == D.DG_OK
    loss_bj = 0.5 * float((T.double() ** 2).sum(1).mean())      # y = 0: block Jacobi alone
    assert loss_trained < 0.5 * loss_bj, (loss_trained, loss_bj)
    res = L.evaluate(he, max_it=20000)
    assert res["mlp"]["converged"] == 6 and res["bj"]["converged"] == 6
    assert np.all(res["mlp"]["relres"] <= 1e-10)
    print(f"mean Arnoldi steps: network {np.mean(res['mlp']['its']):.1f}, block Jacobi "
          f"{np.mean(res['bj']['its']):.1f} (ratio {np.mean(res['mlp']['its']) / np.mean(res['bj']['its']):.3f})")
    h.close()
    he.close()
