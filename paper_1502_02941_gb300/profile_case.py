"""Launch one hot kernel of the solver on the 256x256 P2 workload, for
profilers (a small, self-contained case: ~0.6 GB on the device).

    python -m paper_1502_02941_gb300.profile_case --kernel dots --j 25 --reps 3
    python -m paper_1502_02941_gb300.profile_case --kernel apply64 --reps 3

dots / update: the Arnoldi multi-dot / update kernel of f64 (or --f32) GMRES at
step j on a synthetic basis (dg_profile_kernel); apply64 / apply32 / apply16:
the block-sparse operator apply on the f64 / f32 / bf16 block copy.  Prints the
average CUDA-event time per launch as one JSON line.
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", required=True, choices=["dots", "update", "apply64", "apply32", "apply16"])
    ap.add_argument("--j", type=int, default=25)
    ap.add_argument("--f32", action="store_true", help="f32 Arnoldi kernels (dots / update)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--N", type=int, default=256)
    a = ap.parse_args(argv)

    import torch

    from . import dg as D
    from . import problem
    from . import workloads as W

    cfg = W.config2(method=2, N=a.N)
    h = D.DG(0)
    problem.setup(h, cfg, store=D.DG_STORE_F64 | D.DG_STORE_F32 | D.DG_STORE_BF16, gmres_m=50)
    info = h.info()
    out = {"kernel": a.kernel, "N": a.N, "ne": info.ne, "dofs": info.dofs}
    if a.kernel in ("dots", "update"):
        which = D.DG_PROF_DOTS if a.kernel == "dots" else D.DG_PROF_UPDATE
        out["j"] = a.j
        out["ms"] = h.profile_kernel(which, D.DG_F32 if a.f32 else D.DG_F64, a.j, reps=a.reps)
    else:
        dt = {"apply64": D.DG_F64, "apply32": D.DG_F32, "apply16": D.DG_BF16}[a.kernel]
        td = torch.float64 if dt == D.DG_F64 else torch.float32
        x = torch.randn(info.dofs, dtype=td, device="cuda")
        y = torch.empty_like(x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(a.reps):
            e0.record()
            h.apply(x, dt, y)
            e1.record()
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        out["ms"] = tot / a.reps
    print(json.dumps(out))
    h.close()


if __name__ == "__main__":
    main()
