"""Run the oracle's full FP64 GMRES(50) + block-Jacobi solves of the 256x256
P2 boundary-layer workload (NIPG and SIPG, rel-res 1e-10) and record the
iteration counts and timings in oracle/layer256_p2_oracle_solves.json.

The benchmark's CPU-baseline legs time a bounded slice of the same oracle solve
(assembly, block inverses and a fixed number of iterations) and scale the
per-iteration time by these counts.  This script calls only oracle/ and the
input generators.
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_1502_02941_gb300 import workloads as W  # noqa: E402


def run(method, N=256):
    cfg = W.boundary_layer_p2(method=method, N=N)
    ma = W.structured_mesh(cfg.N)
    m = O.make_mesh(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
    s, kap = O.set_parameter(cfg.method, cfg.k)
    xq = O.quad_points(m, cfg.k, O.VOLUME)
    xb = O.quad_points(m, cfg.k, O.BOUNDARY)
    p = cfg.problem
    t0 = time.time()
    sysm = O.assemble(m, cfg.k, kap, s, 2 * s, p.eps, p.alpha, p.b, p.f(np, xq[..., 0], xq[..., 1]),
                      p.gD(np, xb[..., 0], xb[..., 1]), None, split=False)
    t1 = time.time()
    x, its, relres, ok = O.gmres(m, sysm.A_diag, sysm.A_off, sysm.F, m=50, tol=1e-10, max_it=20000)
    t2 = time.time()
    return {"method": "NIPG" if method == 1 else "SIPG", "N": N, "k": cfg.k, "iterations": its,
            "relres": relres, "converged": ok, "assemble_s": t1 - t0, "gmres_s": t2 - t1}


if __name__ == "__main__":
    out = {"workload": "256x256 split squares, P2, eps=1e-6, b=(1,0), alpha=1, boundary-layer u, "
                       "GMRES(50)+block-Jacobi, rel-res 1e-10",
           "host": os.uname().machine, "solves": [run(1), run(2)]}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "layer256_p2_oracle_solves.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))
