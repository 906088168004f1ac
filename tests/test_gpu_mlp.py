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
    cfg = W.config2(method=2, N=N)
    cfg.k = k
    h = D.DG(0)
    problem.setup(h, cfg, tol=1e-11, gmres_m=30)
    h.precond_setup()
    return h, cfg


@pytest.mark.parametrize("k", [1, 2])
def test_loss_and_gradient_match_oracle(k):
    """GPU loss/gradient (f32 GEMMs, bf16-rounded weights) vs the FP64 oracle
    backpropagation on the same bf16-rounded weights."""
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
    lo, go = M.loss_and_grad(M.bf16_round(theta), X.astype(np.float64), T.astype(np.float64), nb)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    assert np.abs(grad - go).max() <= 2e-5 * np.abs(go).max()
    h.close()


def _oracle_forward_bf16(theta, X, nb):
    """Oracle forward with the kernel's roundings: bf16 weights, inputs and
    hidden activations; f64 arithmetic otherwise."""
    W1, b1, W2, b2, W3, b3, W4, b4 = M.unpack(M.bf16_round(theta), nb)
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
    xstar, _ = h.gmres_solve()
    xk = torch.zeros_like(xstar)
    h.mlp_collect(xstar, xk)
    assert h.mlp_rows() == info.ne
    X = np.zeros((info.ne, M.din_of(nb)), np.float32)
    T = np.zeros((info.ne, nb), np.float32)
    assert D.dg_mlp_get_rows(h.h, X, T, info.ne) == D.DG_OK
    # oracle features from the same GPU residual r = F - A xk = F
    F = _np(h.rhs())
    _, nbr = h.blocks()
    nbr = _np(nbr).astype(np.int64)
    p = cfg.problem
    geo_c = np.zeros((info.ne, 4))
    ma = W.structured_mesh(cfg.N)
    cen = ma.nodes[ma.elems].mean(1)
    geo_c[:, 0] = p.eps
    geo_c[:, 1] = p.b[0] + p.b[1] * cen[:, 0] + p.b[2] * cen[:, 1]
    geo_c[:, 2] = p.b[3] + p.b[4] * cen[:, 0] + p.b[5] * cen[:, 1]
    geo_c[:, 3] = p.alpha
    Xo, so = M.features(F, nbr, nb, geo_c)
    np.testing.assert_allclose(X, Xo, rtol=2e-6, atol=2e-6)
    zbj = _np(h.precond_apply(h.rhs(), D.DG_F64))
    To = ((_np(xstar) - zbj).reshape(info.ne, nb)) / so[:, None]
    np.testing.assert_allclose(T, To, rtol=1e-5, atol=1e-5 * np.abs(To).max())
    h.close()


def test_flexible_gmres_with_mlp_converges():
    """A randomly initialised network is a poor but valid preconditioner:
    flexible GMRES still reaches the tolerance (oracle-independent check of the
    f64 residual), falling back to block Jacobi if it stalls."""
    h, cfg = _handle(2, N=8)
    h.mlp_init(seed=1)
    h.set_params(precond=D.DG_PRECOND_MLP)
    x, info = h.gmres_solve()
    assert info.status == D.DG_OK and info.relres <= 1e-11
    h.set_params(precond=D.DG_PRECOND_BLOCK_JACOBI)
    xb, ib = h.gmres_solve()
    assert np.abs(_np(x) - _np(xb)).max() <= 1e-8 * np.abs(_np(xb)).max()
    h.close()


def test_training_reduces_loss():
    h, cfg = _handle(2, N=12)
    h.mlp_init(seed=2)
    xstar, _ = h.gmres_solve()
    for its in (5, 15, 40):
        h.set_params(max_it=its)
        xk, _ = h.gmres_solve(raise_on_nonconv=False)
        h.mlp_collect(xstar, xk)
    loss = h.mlp_train(300, batch_rows=1024, lr=2e-3, seed=5)
    assert loss[-20:].mean() < 0.5 * loss[:5].mean()
    h.close()
