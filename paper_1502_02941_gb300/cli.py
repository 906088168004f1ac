"""Command-line solve of one workload through libdg.

    python -m paper_1502_02941_gb300.cli --workload layer --N 256 --method 2 --solver gmres
    python -m paper_1502_02941_gb300.cli --workload bump --N 64 --solver mixed-bf16
    python -m paper_1502_02941_gb300.cli --workload bump --solver gmres-ir-f32 --max-it 400000
    python -m paper_1502_02941_gb300.cli --workload bump --solver gmres-ir-f32 --precond schwarz
    python -m paper_1502_02941_gb300.cli --workload tanh-u2 --solver newton

Workloads: sine (8x8 split squares, P1 SIPG, u = sin(pi x) sin(pi y)), layer
(256x256, P2, eps = 1e-6 boundary layer), bump (512x512, P3, rotating flow,
Gaussian bump, Neumann right/top), tanh-u2 (the paper's non-linear example:
8x8, P1, tanh layer with r(u) = u^2; --k sets the degree); --N changes the mesh
size.  The newton solver applies to tanh-u2.

Prints one JSON line with sizes, iterations, relative residual, L2 error (when
the workload has an exact solution) and wall time of the solve.
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="layer", choices=["sine", "layer", "bump", "tanh-u2"])
    ap.add_argument("--k", type=int, default=None, help="degree (tanh-u2)")
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--method", type=int, default=None, help="1 NIPG, 2 SIPG, 3 IIPG")
    ap.add_argument("--solver", default="gmres",
                    choices=["gmres", "dense", "mixed-bf16", "mixed-f32", "gmres-ir-bf16", "gmres-ir-f32",
                             "newton"])
    ap.add_argument("--precond", default="block-jacobi", choices=["block-jacobi", "schwarz", "none"])
    ap.add_argument("--m", type=int, default=50)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--max-it", type=int, default=20000)
    ap.add_argument("--repeat", type=int, default=1)
    a = ap.parse_args(argv)

    import torch

    from . import dg as D
    from . import problem
    from . import workloads as W

    if a.workload == "sine":
        cfg = W.sine_8x8()
    elif a.workload == "layer":
        cfg = W.boundary_layer_p2(method=a.method or 2, N=a.N or 256)
    elif a.workload == "tanh-u2":
        cfg = W.tanh_nonlinear(N=a.N or 8, k=a.k or 1, method=a.method or 2)
    else:
        cfg = W.gaussian_bump_p3(N=a.N or 512)
    if (a.solver == "newton") != bool(cfg.problem.reaction):
        ap.error("--solver newton goes with the non-linear workload tanh-u2, and only there")
    if a.N and a.workload == "sine":
        cfg.N = a.N
    if a.method:
        cfg.method = a.method
    store = D.DG_STORE_F64
    if a.solver.endswith("bf16"):
        store |= D.DG_STORE_BF16
    elif a.solver.endswith("f32"):
        store |= D.DG_STORE_F32
    h = D.DG(0)
    pc = {"block-jacobi": D.DG_PRECOND_BLOCK_JACOBI, "schwarz": D.DG_PRECOND_SCHWARZ,
          "none": D.DG_PRECOND_NONE}[a.precond]
    problem.setup(h, cfg, store=store, gmres_m=a.m, tol=a.tol, max_it=a.max_it, precond=pc)
    h.precond_setup(pc)
    info = h.info()
    out = {}
    for _ in range(a.repeat):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if a.solver == "dense":
            x = h.dense_solve()
            si = None
        elif a.solver == "gmres":
            x, si = h.gmres_solve(raise_on_nonconv=False)
        elif a.solver == "newton":
            p, c = cfg.problem.reaction
            x, si = h.newton_solve(p=p, c=c, max_newton=50, lin_tol=min(1e-2, 100 * a.tol), raise_on_nonconv=False)
        elif a.solver.startswith("mixed"):
            dt = D.DG_BF16 if a.solver == "mixed-bf16" else D.DG_F32
            x, si = h.mixed_solve(dt, inner_m=a.m, inner_tol=1e-2 if dt == D.DG_BF16 else 1e-4, max_outer=60,
                                  raise_on_nonconv=False)
        else:
            dt = D.DG_BF16 if a.solver == "gmres-ir-bf16" else D.DG_F32
            x, si = h.gmres_ir_solve(dt, inner_m=a.m, inner_tol=1e-2 if dt == D.DG_BF16 else 1e-4, max_outer=5000,
                                     raise_on_nonconv=False)
        torch.cuda.synchronize()
        out["seconds"] = time.perf_counter() - t0
    if si is not None:
        out.update(iterations=si.iterations, outer=si.outer, relres=si.relres, status=D.status_name(si.status))
    if cfg.problem.exact is not None:
        l2, hmax = h.l2_error(x, problem.exact_at_error_points(h, cfg.problem))
        out.update(l2_error=l2, h_max=hmax)
    out.update(workload=a.workload, N=cfg.N, k=cfg.k, method=cfg.method, ne=info.ne, dofs=info.dofs,
               solver=a.solver, precond=a.precond)
    print(json.dumps(out))
    h.close()


if __name__ == "__main__":
    main()
