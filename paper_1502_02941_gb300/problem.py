"""Set up a workload (paper_1502_02941_gb300.workloads.Config) on a DG handle.

Problem data f, gD, gN are evaluated at the library's own quadrature points on
the device (the role of the paper's vectorised sub-functions fsource, DBCexact
and NBCexact); everything else is a call into libdg.
"""
from __future__ import annotations

import numpy as np

from . import dg as D
from . import workloads as W


def mesh_for(cfg: W.Config) -> W.MeshArrays:
    return W.structured_mesh(cfg.N, cfg.problem.neumann_sides)


def problem_data(h: D.DG, prob: W.Problem):
    """f at the volume points, gD / gN at the boundary points (device tensors)."""
    torch = h.torch
    xq = h.quad_points(D.DG_POINTS_VOLUME)
    f = prob.f(torch, xq[..., 0], xq[..., 1]).contiguous()
    xb = h.quad_points(D.DG_POINTS_BOUNDARY)
    nrm, _ = h.boundary_info()
    gD = prob.gD(torch, xb[..., 0], xb[..., 1]).contiguous()
    gN = prob.gN(torch, xb[..., 0], xb[..., 1], nrm[:, None, 0], nrm[:, None, 1]).contiguous()
    return f, gD, gN


def eps_data(h: D.DG, prob: W.Problem):
    """A variable diffusion coefficient (the paper's fdiff) at the volume and
    face points (device tensors), or (None, None) for a constant eps."""
    if prob.eps_fn is None:
        return None, None
    torch = h.torch
    xq = h.quad_points(D.DG_POINTS_VOLUME)
    xf = h.quad_points(D.DG_POINTS_FACE)
    return (prob.eps_at(torch, xq[..., 0], xq[..., 1]).contiguous(),
            prob.eps_at(torch, xf[..., 0], xf[..., 1]).contiguous())


def setup(h: D.DG, cfg: W.Config, store=D.DG_STORE_F64, mesh: W.MeshArrays | None = None,
          assemble: bool = True, **params):
    ma = mesh if mesh is not None else mesh_for(cfg)
    h.mesh_upload(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
    h.set_params(method=cfg.method, degree=cfg.k, sigma_int=float(cfg.sigma or 0.0), store=store, **params)
    data = problem_data(h, cfg.problem)
    if assemble:
        p = cfg.problem
        eq, ef = eps_data(h, p)
        h.assemble(p.eps, p.alpha, p.b, *data, eps_q=eq, eps_f=ef)
    return ma, data


def setup_batch(h: D.DG, cfgs, ma: W.MeshArrays, elem_start, coeffs, store=D.DG_STORE_F64, **params):
    """Upload a concatenated batch mesh, declare the instances, evaluate each
    instance's f at its own volume points (gD = gN = 0: homogeneous Dirichlet
    data on every instance) and assemble all instances in one pass."""
    torch = h.torch
    k = cfgs[0].k
    if any(c.k != k for c in cfgs) or any(c.method != cfgs[0].method for c in cfgs):
        raise ValueError("the instances of one batch share the degree and the method")
    h.mesh_upload(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
    h.set_params(method=cfgs[0].method, degree=k, sigma_int=0.0, store=store, **params)
    h.batch_setup(elem_start, coeffs)
    xq = h.quad_points(D.DG_POINTS_VOLUME)
    f = torch.empty(xq.shape[:2], dtype=torch.float64, device=xq.device)
    for i, c in enumerate(cfgs):
        a, b = int(elem_start[i]), int(elem_start[i + 1])
        f[a:b] = c.problem.f(torch, xq[a:b, :, 0], xq[a:b, :, 1])
    h.assemble(0.0, 0.0, (0,) * 6, f.contiguous(), None, None)
    return f


def exact_at_error_points(h: D.DG, prob: W.Problem):
    xe = h.quad_points(D.DG_POINTS_ERROR)
    return prob.u(h.torch, xe[..., 0], xe[..., 1]).contiguous()
