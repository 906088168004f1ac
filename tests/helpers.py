"""Shared test glue: run the oracle on a workload (inputs from workloads.py)."""
import os
from dataclasses import dataclass

import numpy as np

import oracle as O
from paper_1502_02941_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden_sections(name):
    sec, out = None, {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line[0].isalpha():
                sec = line
                out[sec] = []
                continue
            out.setdefault(sec, []).append([float(v) for v in line.split()])
    return {k: np.array(v) for k, v in out.items()}


@dataclass
class OracleRun:
    mesh: O.Mesh
    k: int
    system: O.System
    kappa: float
    sigma: float


def oracle_system(ma: W.MeshArrays, k: int, method: int, prob: W.Problem, sigma=None,
                  literal_rhs=False, split=True, b0=1.0) -> OracleRun:
    m = O.make_mesh(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
    s, kap = O.set_parameter(method, k)
    if sigma is not None:
        s = sigma
    xq = O.quad_points(m, k, O.VOLUME)
    xb = O.quad_points(m, k, O.BOUNDARY)
    nrm = O.boundary_normals(m)
    f = prob.f(np, xq[..., 0], xq[..., 1])
    gD = prob.gD(np, xb[..., 0], xb[..., 1])
    gN = prob.gN(np, xb[..., 0], xb[..., 1], nrm[:, None, 0], nrm[:, None, 1])
    ev = ee = None
    if prob.eps_fn is not None:   # variable diffusion: eps at the volume and edge points
        ev = prob.eps_at(np, xq[..., 0], xq[..., 1])
        xe = O.quad_points(m, k, O.EDGES)
        ee = prob.eps_at(np, xe[..., 0], xe[..., 1])
    sysm = O.assemble(m, k, kap, s, 2 * s, prob.eps, prob.alpha, prob.b, f, gD, gN,
                      literal_rhs=literal_rhs, split=split, b0=b0, eps_vol=ev, eps_edge=ee)
    return OracleRun(m, k, sysm, kap, s)


def oracle_direct(run: OracleRun):
    A = O.dense_matrix(run.mesh, run.system.A_diag, run.system.A_off)
    return np.linalg.solve(A, run.system.F)


def oracle_l2(run: OracleRun, coef, prob: W.Problem):
    xe = O.quad_points(run.mesh, run.k, O.ERROR)
    return O.l2_error(run.mesh, run.k, coef, prob.u(np, xe[..., 0], xe[..., 1]))
