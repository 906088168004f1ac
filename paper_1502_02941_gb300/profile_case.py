"""Launch one hot kernel of the solver on the 256x256 P2 workload (or, with
--p3, the P3 Gaussian bump; --N 512 holds ~3 GB), for profilers (a small,
self-contained case: ~0.6 GB on the device).

    python -m paper_1502_02941_gb300.profile_case --kernel dots --j 25 --reps 3
    python -m paper_1502_02941_gb300.profile_case --kernel apply64 --reps 3
    python -m paper_1502_02941_gb300.profile_case --kernel step --reps 1

dots / update: the Arnoldi multi-dot / update kernel of f64 (or --f32) GMRES at
step j on a synthetic basis (dg_profile_kernel); mlp: the learned
preconditioner's tensor-core inference (dg_mlp_forward) on one feature row
per element (131072 rows); train: Adam steps of the learned preconditioner on
8192-row batches (ms per step; its GEMMs run on the tensor cores); bsolve: one batched f32 GMRES-based refinement
(Schwarz) of the P2 instances among the first --batch instances of the
batched workload; apply64 / apply32 / apply16:
the block-sparse operator apply on the f64 / f32 / bf16 block copy (timed by
dg_profile_kernel around the bare launch, L2 flushed by reads before each); assemble:
one assembly; step: the benchmark's step (mesh upload, assembly, block-Jacobi
set-up and f64 GMRES(50) to 1e-10 for NIPG and SIPG) after one untimed step,
inside an NVTX range "timed_steps".  Prints the average CUDA-event time per
launch (per step) as one JSON line.
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", required=True,
                    choices=["dots", "update", "apply64", "apply32", "apply16", "assemble", "step", "mlp",
                             "bsolve", "train"])
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--j", type=int, default=25)
    ap.add_argument("--f32", action="store_true", help="f32 Arnoldi kernels (dots / update)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--N", type=int, default=256)
    ap.add_argument("--p3", action="store_true",
                    help="the P3 Gaussian-bump workload on N x N split squares instead of the P2 boundary layer")
    a = ap.parse_args(argv)

    import torch

    from . import dg as D
    from . import problem
    from . import workloads as W

    cfg = W.gaussian_bump_p3(N=a.N) if a.p3 else W.boundary_layer_p2(method=2, N=a.N)
    h = D.DG(0)
    if a.kernel == "bsolve":
        cfgs, ma, starts, coeffs = W.batch_by_degree("batched", a.batch)[2]
        problem.setup_batch(h, cfgs, ma, starts, coeffs, store=D.DG_STORE_F64 | D.DG_STORE_F32, gmres_m=50,
                            tol=1e-10, max_it=20000, precond=D.DG_PRECOND_SCHWARZ)
        h.precond_setup(D.DG_PRECOND_SCHWARZ)
        tile = h.batch_autotune()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(a.reps):
            e0.record()
            _, its, _, st = h.batch_gmres_ir_solve(D.DG_F32, inner_m=32, inner_tol=1e-3, max_outer=1000)
            e1.record()
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        print(json.dumps({"kernel": "bsolve", "instances": len(cfgs), "dofs": h.info().dofs, "tile": tile,
                          "ms": tot / a.reps, "its_max": int(its.max()), "converged": int((st == 0).sum())}))
        h.close()
        return
    if a.kernel == "step":
        ma = W.structured_mesh(a.N)
        problem.setup(h, cfg, mesh=ma, assemble=False)
        f, gD, gN = problem.problem_data(h, cfg.problem)
        p = cfg.problem
        x = torch.empty(h.info().dofs, dtype=torch.float64, device="cuda")

        def step():
            for method in (1, 2):
                h.mesh_upload(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
                h.set_params(method=method, degree=2, sigma_int=0.0, store=D.DG_STORE_F64, gmres_m=50, tol=1e-10,
                             max_it=20000)
                h.assemble(p.eps, p.alpha, p.b, f, gD, gN)
                h.precond_setup()
                h.gmres_solve(x=x)

        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_steps")
        e0.record()
        for _ in range(a.reps):
            step()
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"kernel": "step", "N": a.N, "ms": e0.elapsed_time(e1) / a.reps}))
        h.close()
        return
    problem.setup(h, cfg, store=D.DG_STORE_F64 | D.DG_STORE_F32 | D.DG_STORE_BF16, gmres_m=50)
    info = h.info()
    out = {"kernel": a.kernel, "N": a.N, "ne": info.ne, "dofs": info.dofs}
    if a.kernel == "assemble":
        p = cfg.problem
        data = problem.problem_data(h, p)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(a.reps):
            e0.record()
            h.assemble(p.eps, p.alpha, p.b, *data)
            e1.record()
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        out["ms"] = tot / a.reps
    elif a.kernel == "mlp":
        h.mlp_init(seed=3)
        rows = info.ne
        din = 4 * info.nb + 8
        X = torch.randn((rows, din), dtype=torch.float32, device="cuda")
        Y = torch.empty((rows, info.nb), dtype=torch.float32, device="cuda")
        h.check(D.dg_mlp_forward(h.h, X, rows, Y))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(a.reps):
            e0.record()
            h.check(D.dg_mlp_forward(h.h, X, rows, Y))
            e1.record()
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        out["ms"] = tot / a.reps
        out["rows"] = rows
        out["tflops"] = 2.0 * rows * (32 * 128 + 2 * 128 * 128 + 128 * 16) / (out["ms"] / 1e3) / 1e12
    elif a.kernel == "train":
        # training rows from a short GMRES run, then Adam steps of 8192 rows
        # (the GEMMs of each step on the tensor cores)
        h.mlp_init(seed=3)
        h.set_params(max_it=10)
        xk, _ = h.gmres_solve(raise_on_nonconv=False)
        h.mlp_collect(xk)
        h.mlp_train(2, batch_rows=8192)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = 10 * a.reps
        e0.record()
        h.mlp_train(steps, batch_rows=8192)
        e1.record()
        e1.synchronize()
        out["ms"] = e0.elapsed_time(e1) / steps
        out["batch_rows"] = 8192
    elif a.kernel in ("dots", "update"):
        which = D.DG_PROF_DOTS if a.kernel == "dots" else D.DG_PROF_UPDATE
        out["j"] = a.j
        out["ms"] = h.profile_kernel(which, D.DG_F32 if a.f32 else D.DG_F64, a.j, reps=a.reps)
    else:
        # the bare launch between CUDA events inside the library, L2 flushed by reads before each
        dt = {"apply64": D.DG_F64, "apply32": D.DG_F32, "apply16": D.DG_BF16}[a.kernel]
        out["ms"] = h.profile_kernel(D.DG_PROF_APPLY, dt, 0, reps=a.reps)
    print(json.dumps(out))
    h.close()


if __name__ == "__main__":
    main()
