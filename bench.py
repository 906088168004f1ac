#!/usr/bin/env python
"""Benchmark of the DG hot path on one GB300 (or N replicas).

Workload: the 256x256 split-square mesh (131072 triangles), P2 (786432 dofs),
eps = 1e-6, b = (1,0), alpha = 1, boundary-layer manufactured solution,
Dirichlet data on all sides; NIPG and SIPG with upwinding; GMRES(50) with
block-Jacobi preconditioning to relative residual 1e-10 (f64).

One step = for each of NIPG and SIPG: mesh upload + device geometry/adjacency,
assembly of the block operator and F, block-Jacobi set-up, GMRES solve.  The
metric is solves/s (2 solves per step).  `value` has the problem data (f, gD,
gN at the quadrature points) resident in HBM; `e2e` copies them from pinned
host memory every step and reads the solution back.

Also reported: the f64 operator apply against the HBM roofline (CUDA events,
same stream), the oracle's CPU time for the same solve (bounded sample), clocks
sampled during the timed region, and the number of kernels launched.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s to rel-res 1e-10, learned+mixed vs plain FP64 GMRES; apply HBM GB/s"
WORKLOAD = "boundary layer: 256x256 split squares (131072 triangles), P2 (786432 dofs), NIPG+SIPG, eps=1e-6, " \
           "b=(1,0), alpha=1, boundary-layer u, all Dirichlet, GMRES(50)+block-Jacobi f64 to rel-res 1e-10"
N_MESH, DEGREE = 256, 2
METHODS = (1, 2)   # NIPG, SIPG
SMS, SM_MAX_GHZ, FP64_FMA_PER_CLK_SM = 152, 2.07, 2   # GB300: FP64 is 1/64 of FP32 per SM
INNER_M = 32   # restart length of the low-precision inner GMRES


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and learned sections")
    ap.add_argument("--batch-instances", type=int, default=1024)
    ap.add_argument("--learned-instances", type=int, default=16, help="training instances")
    ap.add_argument("--learned-eval", type=int, default=128, help="unseen instances evaluated")
    ap.add_argument("--learned-steps", type=int, default=4000)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"dg_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# roofline inputs
# ---------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profile_traffic(name):
    """dram bytes per launch recorded in profiles/<name>.md ('dram_bytes_per_launch: X')."""
    p = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(p):
        return None
    for line in open(p):
        if line.strip().startswith("dram_bytes_per_launch:"):
            try:
                return float(line.split(":", 1)[1].split()[0])
            except ValueError:
                return None
    return None


def apply_bytes(ne, n_interior, nb, s_a, s_x):
    """Algorithmic bytes of one apply: nonzero blocks, x read once, y written once,
    3 neighbour ids per element."""
    blocks = ne + 2 * n_interior
    return blocks * nb * nb * s_a + ne * nb * (s_x + s_x) + 12 * ne


# ---------------------------------------------------------------------------
# batched and learned sections (wall time bracketed by CUDA events on the
# current stream; the library's stream is a blocking stream, so the events
# bracket its work)
# ---------------------------------------------------------------------------
def _events_time(stream, fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, out


BATCH_RUNS = (
    # name, solver, preconditioner, inner precision, inner restart length, inner tolerance, outer cap
    ("f32_gmres_ir_schwarz", "gmres_ir", "schwarz", "f32", 32, 1e-3, 1000),
    ("f32_gmres_ir", "gmres_ir", "bj", "f32", 32, 1e-3, 1000),
    ("f64", "refine", "bj", "f64", 50, 1e-4, 60),
)


def batched_section(local, stream, n_inst, runs=BATCH_RUNS):
    """Instances 0..n_inst-1 of the batched workload (N uniform in [16,128], P1
    or P2 drawn per instance, random coefficients): one batch per degree, the
    two batches solved together in one group call (concurrently, each on its
    own stream), every instance to rel-res 1e-10: f64 FGMRES around batched f32
    GMRES(32) inner solves (GMRES-based refinement) with the Schwarz or the
    block-Jacobi preconditioner, against plain batched f64 GMRES(50) with block
    Jacobi (the plain FP64 baseline)."""
    import numpy as np
    from paper_1502_02941_gb300 import dg as D, problem, workloads as W
    t0 = time.perf_counter()
    groups = W.batch_by_degree("batched", n_inst)
    out = {"workload": f"{n_inst} instances of the batched workload: N in [16,128], k in {{1,2}} drawn per instance, "
                       "eps log-uniform [1e-6,1e-1], |b| U[0,1], alpha U[0,1], 4-Gaussian f; SIPG, homogeneous "
                       "Dirichlet; one batch per degree, both batches in one group call",
           "instances": n_inst, "batches": {}}
    hs, ids = [], []
    for k, (cfgs, ma, starts, coeffs) in groups.items():
        h = D.DG(local)
        problem.setup_batch(h, cfgs, ma, starts, coeffs, store=D.DG_STORE_F64 | D.DG_STORE_F32, gmres_m=50,
                            tol=1e-10, max_it=20000, precond=D.DG_PRECOND_SCHWARZ)
        h.precond_setup(D.DG_PRECOND_SCHWARZ)
        info = h.info()
        tile = h.batch_autotune()
        out["batches"][f"P{k}"] = {"instances": len(cfgs), "ne": info.ne, "dofs": info.dofs, "tile": tile}
        hs.append(h)
        ids.append([int(c.name.split("inst")[1]) for c in cfgs])
    out["setup_s"] = time.perf_counter() - t0
    out["dofs_total"] = sum(b["dofs"] for b in out["batches"].values())
    for name, solver, pc, inner, m_in, tol_in, max_outer in runs:
        for h in hs:
            h.set_params(precond=D.DG_PRECOND_SCHWARZ if pc == "schwarz" else D.DG_PRECOND_BLOCK_JACOBI)
        dt = D.DG_F64 if inner == "f64" else D.DG_F32
        sec, res = _events_time(stream, lambda: D.batch_group(hs, solver, dt, inner_m=m_in, inner_tol=tol_in,
                                                               max_outer=max_outer, raise_on_nonconv=False))
        its = np.concatenate([r[1] for r in res])
        rr = np.concatenate([r[2] for r in res])
        st = np.concatenate([r[3] for r in res])
        inst = np.concatenate([np.array(i) for i in ids])
        conv = st == 0
        out[name] = {"solver": "f64 FGMRES(50) around f32 GMRES(32) inner solves" if solver == "gmres_ir"
                     else "batched f64 GMRES(50)", "preconditioner": "schwarz" if pc == "schwarz" else "block-jacobi",
                     "seconds": sec, "solves_per_s": n_inst / sec, "converged": int(conv.sum()),
                     "converged_per_s": int(conv.sum()) / sec, "its_median": int(np.median(its)),
                     "its_max": int(its.max()),
                     "relres_max_converged": float(rr[conv].max()) if conv.any() else None,
                     "not_converged": sorted(int(i) for i in inst[~conv])}
    for h in hs:
        h.close()
    base = out.get("f64")
    if base:
        for name in out:
            if isinstance(out[name], dict) and "converged_per_s" in out[name] and name != "f64":
                out[name]["converged_per_s_vs_f64"] = out[name]["converged_per_s"] / max(base["converged_per_s"],
                                                                                        1e-12)
    return out


def bump512_section(local, stream, inner_m=32, inner_tol=1e-3):
    """The mixed-precision workload of the 512x512 split squares (524288
    triangles), P3 (5.24 M unknowns): SIPG, eps = 1e-3, rotating b, alpha = 0.1,
    Gaussian-bump solution, Dirichlet left/bottom and Neumann right/top; one
    solve to rel-res 1e-10 by f64 FGMRES(50) around f32 GMRES inner solves with
    the Schwarz preconditioner (GMRES-based refinement), timed after an untimed
    set-up; the relative residual is re-measured with the f64 apply."""
    import torch
    from paper_1502_02941_gb300 import dg as D, problem, workloads as W
    c = W.gaussian_bump_p3(N=512)
    h = D.DG(local)
    t0 = time.perf_counter()
    problem.setup(h, c, store=D.DG_STORE_F64 | D.DG_STORE_F32, gmres_m=50, tol=1e-10, max_it=400000,
                  precond=D.DG_PRECOND_SCHWARZ)
    h.precond_setup(D.DG_PRECOND_SCHWARZ)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = h.info()
    sec, (x, si) = _events_time(stream, lambda: h.gmres_ir_solve(D.DG_F32, inner_m=inner_m, inner_tol=inner_tol,
                                                                 max_outer=5000, raise_on_nonconv=False))
    F = h.rhs()
    rr = (torch.linalg.norm(F - h.apply(x)) / torch.linalg.norm(F)).item()
    l2, _ = h.l2_error(x, problem.exact_at_error_points(h, c.problem))
    h.close()
    return {"workload": "512x512 split squares (524288 triangles), P3 (5242880 dofs), SIPG, eps=1e-3, rotating b, "
                        "alpha=0.1, Gaussian bump, Dirichlet left/bottom, Neumann right/top",
            "solver": f"f64 FGMRES(50) around f32 GMRES({inner_m}) inner solves to {inner_tol:g} or 8 cycles, "
                      "Schwarz preconditioner", "setup_s": setup_s, "seconds": sec, "solves_per_s": 1.0 / sec,
            "inner_iterations": si.iterations, "outer": si.outer, "relres": si.relres, "relres_check": rr,
            "converged": si.status == 0, "l2_error": l2, "dofs": info.dofs}


def nonlinear_section(local, stream):
    """The paper's non-linear example (tanh layer, eps = 1e-6, b = (1,2)/sqrt(5),
    alpha = 1, r(u) = u^2, SIPG) on 256x256 split squares with P2: Newton to
    ||Res|| <= 1e-10 ||F||, each correction by GMRES(50) + block Jacobi on the
    Jacobian to 1e-8; and the H / HJ kernel alone."""
    import torch
    from paper_1502_02941_gb300 import dg as D, problem, workloads as W
    c = W.tanh_nonlinear(N=256, k=2)
    h = D.DG(local)
    problem.setup(h, c, mesh=W.structured_mesh(c.N), gmres_m=50, tol=1e-10, max_it=20000)
    info = h.info()
    h.newton_solve(p=2, c=1.0, max_newton=20, lin_tol=1e-8)            # warm-up
    sec, (x, ni) = _events_time(stream, lambda: h.newton_solve(p=2, c=1.0, max_newton=20, lin_tol=1e-8))
    l2, _ = h.l2_error(x, problem.exact_at_error_points(h, c.problem))
    H = torch.empty(info.dofs, dtype=torch.float64, device=x.device)
    HJ = torch.empty((info.ne, 6, 6), dtype=torch.float64, device=x.device)
    reps = 20
    for _ in range(3):
        D.dg_nonlinear_global(h.h, 2, 1.0, x, H, HJ)
    ksec, _ = _events_time(stream, lambda: [D.dg_nonlinear_global(h.h, 2, 1.0, x, H, HJ) for _ in range(reps)])
    h.close()
    return {"workload": "the paper's non-linear example (tanh layer, r(u) = u^2, eps = 1e-6, b = (1,2)/sqrt(5), "
                        "alpha = 1, SIPG) on 256x256 split squares (131072 triangles), P2 (786432 dofs)",
            "seconds": sec, "newton_steps": ni.outer, "gmres_steps": ni.iterations, "relres": ni.relres,
            "converged": ni.status == 0, "l2_error": l2,
            "k_nonlin_ms": ksec / reps * 1e3, "k_nonlin_elements_per_s": info.ne * reps / ksec}


LEARNED_RUNS = (
    # name, preconditioner, inner precision (f64: batched f64 GMRES(50); f32: f32 inner solves + f64 refinement)
    ("bj_f64", "bj", "f64"), ("schwarz_f64", "schwarz", "f64"), ("mlp_f64", "mlp", "f64"),
    ("bj_f32_refined", "bj", "f32"), ("schwarz_f32_refined", "schwarz", "f32"), ("mlp_f32_refined", "mlp", "f32"),
)


def learned_section(local, stream, n_train, steps, n_eval, chunk=1024, runs=LEARNED_RUNS):
    """Learned preconditioner on the learned workload (64x64 split squares, P2,
    batched-workload coefficients): collect rows from the f64 solves of n_train
    training instances, train on the GPU, then solve n_eval unseen instances
    (in batches of at most `chunk`) with block Jacobi, with the Schwarz
    preconditioner and with the network (flexible GMRES), in f64 and with f32
    inner solves + f64 refinement; steps and time per instance and the ratios
    of the network against both."""
    import numpy as np
    from paper_1502_02941_gb300 import dg as D, learned as L
    pcs = {"bj": D.DG_PRECOND_BLOCK_JACOBI, "schwarz": D.DG_PRECOND_SCHWARZ, "mlp": D.DG_PRECOND_MLP}
    h = D.DG(local)
    t_col, _ = _events_time(stream, lambda: (L.make_batch(h, n_train, 64, first=0, gmres_m=50),
                                             h.mlp_init(seed=7), L.collect(h)))
    rows = h.mlp_rows()
    t_train, (loss, _) = _events_time(stream, lambda: L.train(h, steps=steps))
    theta = h.mlp_get_weights()
    h.close()
    out = {"workload": f"{n_train} training + {n_eval} unseen instances (from instance 1000 on), 64x64 split squares "
                       f"(8192 triangles), P2, solved in batches of at most {chunk} instances",
           "train_instances": n_train, "eval_instances": n_eval, "train_rows": rows, "collect_s": t_col,
           "train_steps": steps, "train_s": t_train, "loss_first": float(loss[0]), "loss_last": float(loss[-1])}
    acc = {name: {"seconds": 0.0, "its": [], "converged": 0} for name, _, _ in runs}
    for first in range(0, n_eval, chunk):
        n = min(chunk, n_eval - first)
        he = D.DG(local)
        L.make_batch(he, n, 64, first=1000 + first, gmres_m=50, store=D.DG_STORE_F64 | D.DG_STORE_F32)
        he.precond_setup(D.DG_PRECOND_SCHWARZ)
        he.mlp_set_weights(theta)
        for name, pc, inner in runs:
            dt = D.DG_F64 if inner == "f64" else D.DG_F32
            he.set_params(precond=pcs[pc], tol=1e-10, max_it=20000)
            # no warm-up solve: at this size graph capture costs milliseconds of a solve of seconds
            sec, (x, its, rr, st) = _events_time(stream, lambda: he.batch_solve(
                dt, inner_m=50, inner_tol=1e-4, max_outer=60, raise_on_nonconv=False))
            a = acc[name]
            a["seconds"] += sec
            a["its"] += [int(v) for v in its]
            a["converged"] += int((st == 0).sum())
        he.close()
    for name, a in acc.items():
        its = np.array(a["its"])
        out[name] = {"seconds": a["seconds"], "solves_per_s": n_eval / a["seconds"], "converged": a["converged"],
                     "its_median": int(np.median(its)), "its_mean": float(its.mean()), "its_max": int(its.max())}
    for base in ("bj", "schwarz"):
        for inner in ("f64", "f32_refined"):
            m, b = out.get(f"mlp_{inner}"), out.get(f"{base}_{inner}")
            if m and b:
                out[f"its_ratio_mlp_vs_{base}_{inner}"] = m["its_mean"] / b["its_mean"]
                out[f"time_ratio_mlp_vs_{base}_{inner}"] = m["seconds"] / b["seconds"]
    return out


# ---------------------------------------------------------------------------
# CPU baseline (the oracle), bounded sample
# ---------------------------------------------------------------------------
ORACLE_ITERS = 50   # one full GMRES(50) restart cycle per method: the MGS cost averaged over j = 0..49


def cpu_info():
    """Host cores visible to this process and the CPU model name."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.strip().lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"nproc": cores, "cpu_model": model or platform.processor() or platform.machine()}


def oracle_sample(gpu_its, iters=ORACLE_ITERS, omp=False):
    """Time the oracle's assembly + block inverses + `iters` GMRES iterations of
    each method and scale the per-iteration time to `gpu_its` (iterations the
    same algorithm needs) -> estimated oracle solves/s.  omp: the oracle's
    all-cores timing build (OpenMP loops), else the serial build.  Returns
    (solves/s, per-method detail, threads used)."""
    import numpy as np

    import oracle as O
    from paper_1502_02941_gb300 import workloads as W
    O.set_openmp(omp)
    try:
        threads = O.num_threads()
        total = 0.0
        detail = []
        for method, its in zip(METHODS, gpu_its):
            cfg = W.boundary_layer_p2(method=method, N=N_MESH)
            ma = W.structured_mesh(cfg.N)
            p = cfg.problem
            t0 = time.perf_counter()
            m = O.make_mesh(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
            s, kap = O.set_parameter(cfg.method, cfg.k)
            xq = O.quad_points(m, cfg.k, O.VOLUME)
            xb = O.quad_points(m, cfg.k, O.BOUNDARY)
            sysm = O.assemble(m, cfg.k, kap, s, 2 * s, p.eps, p.alpha, p.b, p.f(np, xq[..., 0], xq[..., 1]),
                              p.gD(np, xb[..., 0], xb[..., 1]), None, split=False)
            t1 = time.perf_counter()
            _, done, _, _ = O.gmres(m, sysm.A_diag, sysm.A_off, sysm.F, m=50, tol=1e-10, max_it=iters)
            t2 = time.perf_counter()
            per_it = (t2 - t1) / max(done, 1)
            est = (t1 - t0) + per_it * its
            total += est
            detail.append({"method": "NIPG" if method == 1 else "SIPG", "setup_s": round(t1 - t0, 3),
                           "iterations_timed": done, "per_iteration_ms": round(per_it * 1e3, 3),
                           "iterations_scaled_to": its, "est_solve_s": round(est, 3)})
    finally:
        O.set_openmp(False)
    return len(METHODS) / total, detail, threads


def oracle_all_cores(scale_its):
    """The same sample on the oracle's all-cores build; None if that build is
    unavailable on this host."""
    import oracle as O
    try:
        O.build(openmp=True)
    except Exception as e:   # no OpenMP runtime for this compiler
        return {"unavailable": f"oracle OpenMP build failed: {type(e).__name__}"}
    v, detail, threads = oracle_sample(scale_its, omp=True)
    return {"value": v, "unit": "solves/s", "cores": threads, "kind": "oracle (OpenMP loops, timing build)",
            "sample": f"per method: oracle assembly (serial) + block inverses + {ORACLE_ITERS} GMRES(50) "
                      f"iterations on {threads} threads; per-iteration time scaled to {scale_its} iterations",
            "detail": detail}


def workload_config(world):
    """The `config` both arms report (sizes of the step's workload; no measured values)."""
    ne = 2 * N_MESH * N_MESH
    nb = (DEGREE + 1) * (DEGREE + 2) // 2
    return {"workload": WORKLOAD, "N": N_MESH, "k": DEGREE, "ne": ne, "dofs": ne * nb, "methods": ["NIPG", "SIPG"],
            "gmres_m": 50, "tol": 1e-10,
            "l2_policy": "working set > L2 (blocks 151 MB + Krylov basis 321 MB per solve)",
            "parallelism": f"replicas x{world}"}


def oracle_iteration_counts():
    p = os.path.join(ROOT, "oracle", "layer256_p2_oracle_solves.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return [s["iterations"] for s in d["solves"]], "oracle full solves (oracle/layer256_p2_oracle_solves.json)"
    return None, None


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def reference_arm(args, rank):
    if rank != 0:
        return
    its, src = oracle_iteration_counts()
    if its is None:
        its, src = [2000, 2000], "assumed 2000 iterations per solve (no oracle record)"
    for _ in range(args.warmup):
        oracle_sample(its, iters=1)          # untimed: loads the library and pages the inputs in
    vals = []
    t0 = time.perf_counter()
    details, threads = None, 1
    for _ in range(args.steps):
        v, details, threads = oracle_sample(its)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    host = cpu_info()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(world),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                             "sample": f"per step and method: oracle assembly + block inverses + {ORACLE_ITERS} "
                                       f"GMRES(50) iterations (one restart cycle), per-iteration time scaled to "
                                       f"{its} iterations ({src})",
                             "host": host, "detail": details},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# multi-rank timing (replicas: one independent solve stream per GPU, no
# collective on the data path; the only collectives are these)
# ---------------------------------------------------------------------------
def max_over_ranks(ms, world, device=None):
    """The slowest rank's time in ms; every rank takes part and gets it."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank, world, ms_max):
    """Units all ranks processed per second of the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank)

    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__ as G
    G.build()
    from paper_1502_02941_gb300 import dg as D
    from paper_1502_02941_gb300 import problem
    from paper_1502_02941_gb300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    h = D.DG(local)
    layer = W.boundary_layer_p2(method=METHODS[0], N=N_MESH)
    ma = W.structured_mesh(N_MESH)
    # problem data at the quadrature points (identical for both methods)
    problem.setup(h, layer, mesh=ma, assemble=False)
    f, gD, gN = problem.problem_data(h, layer.problem)
    info = h.info()
    dofs = info.dofs
    x = torch.empty(dofs, dtype=torch.float64, device=dev)
    p = layer.problem
    f_h = f.cpu().pin_memory(); gD_h = gD.cpu().pin_memory(); gN_h = gN.cpu().pin_memory()
    x_h = torch.empty(dofs, dtype=torch.float64).pin_memory()
    h2d = (f_h.numel() + gD_h.numel() + gN_h.numel()) * 8 * len(METHODS) \
        + (ma.nodes.nbytes + ma.elems.nbytes + ma.dirichlet.nbytes + ma.neumann.nbytes) * len(METHODS)
    d2h = dofs * 8 * len(METHODS)

    last = {}

    def step(e2e=False):
        its = []
        for method in METHODS:
            if e2e:
                f.copy_(f_h, non_blocking=True); gD.copy_(gD_h, non_blocking=True); gN.copy_(gN_h, non_blocking=True)
            h.mesh_upload(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
            h.set_params(method=method, degree=DEGREE, sigma_int=0.0, store=D.DG_STORE_F64, gmres_m=50,
                         tol=1e-10, max_it=20000)
            h.assemble(p.eps, p.alpha, p.b, f, gD, gN)
            h.precond_setup()
            _, sinfo = h.gmres_solve(x=x)
            its.append(sinfo.iterations)
            last[method] = (sinfo.iterations, sinfo.relres, sinfo.restarts)
            if e2e:
                x_h.copy_(x, non_blocking=True)
        return its

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(e2e, sampler=None):
        barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        n0 = h.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("e2e_steps" if e2e else "timed_steps")   # lets a profiler select the region
        e0.record(stream)
        for _ in range(args.steps):
            step(e2e)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier()
        clocks = sampler.stop() if sampler else None
        ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        return ms, h.launch_count() - n0, clocks

    sampler = ClockSampler(local)
    ms, launches, clocks = timed(False, sampler)
    ms_e2e, _, _ = timed(True)
    value = whole_job_value(len(METHODS) * args.steps, world, ms)
    e2e_value = whole_job_value(len(METHODS) * args.steps, world, ms_e2e)
    its = [last[m][0] for m in METHODS]

    # ---- mixed precision on the same workload: plain f64 refinement around f32
    # inner GMRES, and f64 FGMRES around f32 / bf16 inner GMRES (GMRES-based
    # refinement; plain refinement around bf16 stalls on this workload)
    def mixed_steps(kind, inner, pc=D.DG_PRECOND_BLOCK_JACOBI):
        store = D.DG_STORE_F64 | (D.DG_STORE_BF16 if inner == D.DG_BF16 else D.DG_STORE_F32)
        # inner GMRES(32) to 1e-3 (f32) / 1e-2 (bf16): the fastest setting of a sweep
        # of restart lengths 16..64 and tolerances 1e-3..1e-6 on this workload
        tol_in = 1e-2 if inner == D.DG_BF16 else 1e-3
        res = {}
        for method in METHODS:
            h.mesh_upload(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
            h.set_params(method=method, degree=DEGREE, sigma_int=0.0, store=store, gmres_m=50, tol=1e-10,
                         max_it=20000, precond=pc)
            h.assemble(p.eps, p.alpha, p.b, f, gD, gN)
            h.precond_setup(pc)
            if kind == "ir":
                _, si = h.mixed_solve(inner, inner_m=INNER_M, inner_tol=tol_in, max_outer=60, x=x,
                                      raise_on_nonconv=False)
            else:
                _, si = h.gmres_ir_solve(inner, inner_m=INNER_M, inner_tol=tol_in, max_outer=300, x=x,
                                         raise_on_nonconv=False)
            res[method] = si
        return res

    mixed = {}
    for name, kind, inner, pc in (("f32", "ir", D.DG_F32, D.DG_PRECOND_BLOCK_JACOBI),
                                  ("f32_gmres_ir", "gir", D.DG_F32, D.DG_PRECOND_BLOCK_JACOBI),
                                  ("bf16_gmres_ir", "gir", D.DG_BF16, D.DG_PRECOND_BLOCK_JACOBI),
                                  ("f32_schwarz", "ir", D.DG_F32, D.DG_PRECOND_SCHWARZ)):
        mixed_steps(kind, inner, pc)   # warm-up (graph capture, workspaces)
        torch.cuda.synchronize()
        m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        m0.record(stream)
        for _ in range(args.steps):
            res = mixed_steps(kind, inner, pc)
        m1.record(stream)
        torch.cuda.synchronize()
        mms = m0.elapsed_time(m1)
        # roofline of the f32 inner iteration (block Jacobi: one apply of the f32 A M^-1 per
        # Arnoldi step, whose diagonal blocks are the identity and not read, then the
        # multi-dot over j+2 vectors and the update over j+1 vectors plus the write, at the
        # mean j = (m-1)/2 of full GMRES(m) cycles)
        inner_steps = sum(r.iterations for r in res.values())
        jm = (INNER_M - 1) / 2.0
        ahat_bytes = apply_bytes(info.ne, info.n_interior, info.nb, 4, 4) - info.ne * info.nb * info.nb * 4
        step_bytes = ahat_bytes + 4.0 * dofs * ((jm + 2) + (jm + 2))
        roof = None
        if inner == D.DG_F32 and pc == D.DG_PRECOND_BLOCK_JACOBI:
            achieved = step_bytes * inner_steps / (mms / args.steps / 1e3) / 1e9
            roof = {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": measured_peaks()[0],
                    "frac": achieved / measured_peaks()[0], "bytes_per_inner_step": step_bytes,
                    "inner_steps_per_step": inner_steps,
                    "note": "algorithmic bytes of the f32 Arnoldi steps only (apply + multi-dot + update at the "
                            "cycle-mean j) over the whole solve time (outer f64 residuals and restarts included)"}
        mixed[name] = {"refinement": "f64 residual correction" if kind == "ir" else "f64 FGMRES outer",
                       "preconditioner": "schwarz" if pc == D.DG_PRECOND_SCHWARZ else "block-jacobi",
                       "inner": f"GMRES({INNER_M}) to {1e-2 if inner == D.DG_BF16 else 1e-3:g} or 8 cycles",
                       "solves_per_s": len(METHODS) * args.steps / (mms / 1e3),
                       "ms_per_solve": mms / (len(METHODS) * args.steps),
                       "inner_iterations": {"NIPG": res[1].iterations, "SIPG": res[2].iterations},
                       "outer": {"NIPG": res[1].outer, "SIPG": res[2].outer},
                       "relres_f64": {"NIPG": res[1].relres, "SIPG": res[2].relres},
                       "converged": all(r.status == 0 for r in res.values()),
                       "speedup_vs_f64": (len(METHODS) * args.steps / (mms / 1e3)) / value}
        if roof:
            mixed[name]["roofline"] = roof

    # ---- kernel timings with CUDA events on the launching stream
    h.mesh_upload(ma.nodes, ma.elems, ma.dirichlet, ma.neumann)
    h.set_params(method=2, degree=DEGREE, sigma_int=0.0, precond=D.DG_PRECOND_BLOCK_JACOBI,
                 store=D.DG_STORE_F64 | D.DG_STORE_F32 | D.DG_STORE_BF16,
                 gmres_m=50, tol=1e-10, max_it=20000)
    h.assemble(p.eps, p.alpha, p.b, f, gD, gN)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    def time_apply(hh, n, dt, reps=30):
        """(kernel ms, ms through the binding): the first from CUDA events around
        the bare launch inside the library (dg_profile_kernel, L2 flushed by a
        read sweep before each launch); the second from events around the public
        call after an L2 flush, which adds the host side of the call (argument
        checks, ctypes) whenever that takes longer than the flush."""
        hh.profile_kernel(D.DG_PROF_APPLY, dt, 0, reps=3)
        kern = hh.profile_kernel(D.DG_PROF_APPLY, dt, 0, reps=reps)
        td = torch.float64 if dt == D.DG_F64 else torch.float32
        xr = torch.randn(n, dtype=td, device=dev)
        yr = torch.empty_like(xr)
        for _ in range(3):
            hh.apply(xr, dt, yr)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(reps):
            flush.sum()   # a read sweep: no dirty lines left for the apply to write back
            a0.record(stream)
            hh.apply(xr, dt, yr)
            a1.record(stream)
            a1.synchronize()
            tot += a0.elapsed_time(a1)
        return kern, tot / reps

    peak, peak_src = measured_peaks()
    # assembly (volume + face integrals + F) alone, f64 blocks and f64+f32+bf16
    assembly = {}
    for name, store in (("f64", D.DG_STORE_F64), ("f64_f32_bf16", D.DG_STORE_F64 | D.DG_STORE_F32 | D.DG_STORE_BF16)):
        h.set_params(store=store)
        h.assemble(p.eps, p.alpha, p.b, f, gD, gN)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        a0.record(stream)
        for _ in range(reps):
            h.assemble(p.eps, p.alpha, p.b, f, gD, gN)
        a1.record(stream)
        torch.cuda.synchronize()
        ams = a0.elapsed_time(a1) / reps
        written = info.ne * 4 * info.nb * info.nb * (8 + (6 if name != "f64" else 0))
        # f64 pipe operations of the entry kernel: per entry of the 4 blocks, 10 volume
        # terms + per face 11 factor terms and 3 per upwind point (k + 2 points)
        ops = info.ne * info.nb * info.nb * (43 + 9 * (DEGREE + 2))
        fp64_ops_peak = SMS * FP64_FMA_PER_CLK_SM * SM_MAX_GHZ * 1e9
        assembly[name] = {"ms": ams, "elements_per_s": info.ne / (ams / 1e3), "bytes_written": written,
                          "GBps_written": written / (ams / 1e3) / 1e9, "fp64_ops": ops,
                          "frac_fp64_peak": ops / (ams / 1e3) / fp64_ops_peak}
    apply = {}
    for name, dt, sa, sx in (("f64", D.DG_F64, 8, 8), ("f32", D.DG_F32, 4, 4), ("bf16", D.DG_BF16, 2, 4)):
        ams, cms = time_apply(h, dofs, dt)
        abytes = apply_bytes(info.ne, info.n_interior, info.nb, sa, sx)
        apply[name] = {"ms": ams, "bytes": abytes, "GBps": abytes / (ams / 1e3) / 1e9,
                       "frac_hbm": abytes / (ams / 1e3) / 1e9 / peak, "ms_via_binding": cms}
    apply["f64"]["fma_per_apply"] = (info.ne + 2 * info.n_interior) * info.nb * info.nb
    # the same kernels on the 512x512 P3 operator (5.24 M unknowns), large enough
    # that launch and tail latency no longer hide the bandwidth
    h3 = D.DG(local)
    bump = W.gaussian_bump_p3(N=512)
    problem.setup(h3, bump, store=D.DG_STORE_F64 | D.DG_STORE_F32 | D.DG_STORE_BF16)
    i3 = h3.info()
    apply_p3 = {}
    for name, dt, sa, sx in (("f64", D.DG_F64, 8, 8), ("f32", D.DG_F32, 4, 4), ("bf16", D.DG_BF16, 2, 4)):
        ams, cms = time_apply(h3, i3.dofs, dt, reps=20)
        abytes = apply_bytes(i3.ne, i3.n_interior, i3.nb, sa, sx)
        apply_p3[name] = {"ms": ams, "bytes": abytes, "GBps": abytes / (ams / 1e3) / 1e9,
                          "frac_hbm": abytes / (ams / 1e3) / 1e9 / peak, "ms_via_binding": cms}
    h3.close()
    jmid = 25
    dots_ms = h.profile_kernel(D.DG_PROF_DOTS, D.DG_F64, jmid)
    upd_ms = h.profile_kernel(D.DG_PROF_UPDATE, D.DG_F64, jmid)
    fp64_peak_tflops = FP64_FMA_PER_CLK_SM * 2 * SMS * SM_MAX_GHZ * 1e9 / 1e12
    dots_flops = 2.0 * (jmid + 2) * dofs
    upd_flops = 2.0 * (jmid + 1) * dofs
    roofline = {"bound": "alu", "kernel": f"k_gm_dots<double> (Arnoldi multi-dot, step j={jmid}, the largest "
                                          "share of the f64 GMRES step)",
                "achieved": dots_flops / (dots_ms / 1e3) / 1e12, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "frac": dots_flops / (dots_ms / 1e3) / 1e12 / fp64_peak_tflops,
                "traffic": profile_traffic("k_gm_dots_f64_layer256_p2"),
                "algorithmic_flops": dots_flops, "algorithmic_bytes": 8.0 * (jmid + 2) * dofs,
                "avg_launch_ms": dots_ms,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (f64 FMA probe measured "
                               "1.19 TFLOP/s); HBM peak for the applies is measured hbm_gbs"}
    kernels = {"k_gm_update<double>": {"ms": upd_ms, "TFLOPs": upd_flops / (upd_ms / 1e3) / 1e12,
                                       "GBps": 8.0 * (jmid + 3) * dofs / (upd_ms / 1e3) / 1e9},
               "k_apply": apply, "k_apply_512x512_P3": apply_p3}

    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(world),
            "solve": {"iterations": {"NIPG": its[0], "SIPG": its[1]},
                      "relres": {"NIPG": last[1][1], "SIPG": last[2][1]}},
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clocks, "roofline": roofline,
            "mixed": mixed, "assembly": assembly, "kernels": kernels, "hbm_peak_GBps": peak}
    if not args.no_extras:
        line["batched"] = batched_section(local, stream, args.batch_instances)
        line["learned"] = learned_section(local, stream, args.learned_instances, args.learned_steps,
                                          args.learned_eval)
        line["nonlinear"] = nonlinear_section(local, stream)
        line["bump512_p3"] = bump512_section(local, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ref_its, _ = oracle_iteration_counts()
        scale_its = ref_its if ref_its else its
        cpu_val, detail, threads = oracle_sample(scale_its)
        line["cpu_baseline"] = {"value": cpu_val, "unit": "solves/s", "cores": threads, "kind": "oracle",
                                "sample": f"per method: oracle assembly + block inverses + {ORACLE_ITERS} GMRES(50) "
                                          f"iterations (one restart cycle); per-iteration time scaled to "
                                          f"{scale_its} iterations",
                                "host": cpu_info(), "detail": detail,
                                "all_cores": oracle_all_cores(scale_its)}
    # the headline figures once more, last in the line (a reader of its tail sees them)
    summ = {"f64_gmres_solves_per_s": value, "e2e_solves_per_s": e2e_value,
            "mixed_solves_per_s": {k: v["solves_per_s"] for k, v in mixed.items()},
            "f32_refined_roofline_frac": mixed.get("f32", {}).get("roofline", {}).get("frac"),
            "apply_512x512_P3_frac_hbm": {k: v["frac_hbm"] for k, v in apply_p3.items()},
            "roofline_frac": roofline["frac"]}
    if "batched" in line:
        b = line["batched"]
        summ["batched"] = {k: {"converged": b[k]["converged"], "seconds": b[k]["seconds"],
                               "converged_per_s": b[k]["converged_per_s"]}
                           for k in b if isinstance(b[k], dict) and "converged_per_s" in b[k]}
    if "learned" in line:
        summ["learned"] = {k: v for k, v in line["learned"].items() if k.startswith(("its_ratio", "time_ratio"))}
    if "bump512_p3" in line:
        summ["bump512_p3"] = {k: line["bump512_p3"][k] for k in ("seconds", "relres_check", "converged")}
    if "cpu_baseline" in line:
        summ["cpu_baseline"] = {"value": line["cpu_baseline"]["value"],
                                "all_cores": line["cpu_baseline"]["all_cores"].get("value")}
    line["summary"] = summ
    if rank == 0:
        print(json.dumps(line))
    h.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
