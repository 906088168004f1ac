"""Glue for the GPU parity tests: run a workload through libdg and through the
oracle on the same seeded inputs, and map between the two bases.

The GPU path uses an orthonormal Dubiner basis, the oracle scaled monomials, so
raw coefficients are never compared.  Per element K the change of basis T_K
(phi_gpu_j = sum_m T_K[m, j] phi_oracle_m) is recovered from values of both
bases at the same physical points; then
    A_gpu(K, L) = T_K^T A_oracle(K, L) T_L,   F_gpu(K) = T_K^T F_oracle(K),
    x_oracle(K) = T_K x_gpu(K).
"""
import numpy as np

import oracle as O
from paper_1502_02941_gb300 import dg as D
from paper_1502_02941_gb300 import problem
from paper_1502_02941_gb300 import workloads as W
from helpers import oracle_system


def gpu_setup(ma: W.MeshArrays, k: int, method: int, prob: W.Problem, sigma=None, store=D.DG_STORE_F64, **params):
    h = D.DG(0)
    cfg = W.Config("t", 0, k, method, prob, sigma=sigma)
    problem.setup(h, cfg, store=store, mesh=ma, **params)
    return h


def basis_change(run, ma: W.MeshArrays, k: int) -> np.ndarray:
    rs, _ = D.dg_reference_rule(D.DG_POINTS_VOLUME, k)
    phig, _, _ = D.dg_reference_basis(k, rs)                           # [Q, nb]
    v = ma.nodes[ma.elems]                                             # [ne, 3, 2]
    xy = v[:, None, 0, :] + rs[None, :, 0, None] * (v[:, None, 1, :] - v[:, None, 0, :]) \
        + rs[None, :, 1, None] * (v[:, None, 2, :] - v[:, None, 0, :])  # [ne, Q, 2]
    ne, Q = xy.shape[0], xy.shape[1]
    _, phio = O.evaluate(run.mesh, k, None, np.repeat(np.arange(ne), Q), xy.reshape(-1, 2), want_basis=True)
    Vo = phio.reshape(ne, Q, -1)                                       # [ne, Q, nb]
    G = np.einsum("kqm,kqn->kmn", Vo, Vo)
    R = np.einsum("kqm,qj->kmj", Vo, phig)
    return np.linalg.solve(G, R)                                       # [ne, nb, nb]


def oracle_blocks(run, ma: W.MeshArrays):
    """Oracle A in the GPU slot layout: [ne, 4, nb, nb] with slot 1+f the
    neighbour across face f (zero on the boundary) and nbr [ne, 3]."""
    m = run.mesh
    Ad, Ao = run.system.A_diag, run.system.A_off
    ne, nb = Ad.shape[0], Ad.shape[1]
    out = np.zeros((ne, 4, nb, nb))
    nbr = -np.ones((ne, 3), np.int64)
    out[:, 0] = Ad
    for f in range(3):
        e = m.elem_edges[:, f]
        Ki, Kj = m.edges[e, 2], m.edges[e, 3]
        K = np.arange(ne)
        interior = Kj >= 0
        own_i = K == Ki
        L = np.where(own_i, Kj, Ki)
        blk = np.where((own_i[:, None, None]), Ao[e, 0], Ao[e, 1])
        out[interior, 1 + f] = blk[interior]
        nbr[interior, f] = L[interior]
    return out, nbr


def to_gpu_basis(T, blocks, nbr):
    """T_K^T B(K, L) T_L for every stored block."""
    out = np.zeros_like(blocks)
    Tt = np.transpose(T, (0, 2, 1))
    out[:, 0] = Tt @ blocks[:, 0] @ T
    for f in range(3):
        L = nbr[:, f]
        ok = L >= 0
        out[ok, 1 + f] = Tt[ok] @ blocks[ok, 1 + f] @ T[L[ok]]
    return out


def oracle_run(ma, k, method, prob, sigma=None, split=True):
    return oracle_system(ma, k, method, prob, sigma=sigma, split=split)


def x_to_oracle(T, xg):
    ne, nb = T.shape[0], T.shape[1]
    return np.einsum("kmj,kj->km", T, xg.reshape(ne, nb)).reshape(-1)


def rel_residual_oracle(run, T, xg):
    xo = x_to_oracle(T, xg)
    r = run.system.F - O.apply(run.mesh, run.system.A_diag, run.system.A_off, xo)
    return np.linalg.norm(r) / np.linalg.norm(run.system.F)
