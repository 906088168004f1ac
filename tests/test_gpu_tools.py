"""The command-line tools of the package run and print their JSON line."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, "-m", *args], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_cli_dense_solve_of_the_8x8_workload():
    out = _run("paper_1502_02941_gb300.cli", "--workload", "sine", "--solver", "dense")
    assert out["ne"] == 128 and out["dofs"] == 384
    assert 0 < out["l2_error"] < 5e-2


@pytest.mark.parametrize("solver", ["gmres", "mixed-f32", "gmres-ir-bf16"])
def test_cli_iterative_solvers(solver):
    out = _run("paper_1502_02941_gb300.cli", "--workload", "layer", "--N", "16", "--solver", solver)
    assert out["status"] == "DG_OK" and out["relres"] <= 1e-10


def test_cli_newton_on_the_papers_nonlinear_example():
    out = _run("paper_1502_02941_gb300.cli", "--workload", "tanh-u2", "--solver", "newton")
    assert out["status"] == "DG_OK" and out["relres"] <= 1e-10 and 1 <= out["outer"] <= 15
    # L2 error and h_max of the paper's driver, against the oracle's Newton solve
    import oracle as O
    from paper_1502_02941_gb300 import workloads as W
    from helpers import oracle_l2, oracle_system
    c = W.tanh_nonlinear()
    run = oracle_system(W.structured_mesh(c.N), c.k, c.method, c.problem)
    v, _, _ = O.newton(run.mesh, run.system, 2, 1.0, tol=1e-12)
    l2o, hmo = oracle_l2(run, v, c.problem)
    assert out["ne"] == 128 and abs(out["l2_error"] - l2o) <= 1e-5 * l2o and abs(out["h_max"] - hmo) <= 1e-15


@pytest.mark.parametrize("kernel", ["dots", "update", "apply32", "apply16", "assemble", "mlp", "train"])
def test_profile_case_kernels(kernel):
    out = _run("paper_1502_02941_gb300.profile_case", "--kernel", kernel, "--N", "32", "--reps", "2")
    assert out["ms"] > 0


def test_profile_hook_times_the_apply_of_each_stored_copy():
    """DG_PROF_APPLY times one bare apply per stored block copy; a copy that is
    not stored is a state error, an unknown dtype an argument error."""
    from paper_1502_02941_gb300 import dg as D
    from paper_1502_02941_gb300 import problem
    from paper_1502_02941_gb300 import workloads as W
    h = D.DG(0)
    problem.setup(h, W.boundary_layer_p2(N=16), store=D.DG_STORE_F64 | D.DG_STORE_F32, gmres_m=20)
    for dt in (D.DG_F64, D.DG_F32):
        assert h.profile_kernel(D.DG_PROF_APPLY, dt, 0, reps=2) > 0
    for dt, st in ((D.DG_BF16, D.DG_ERR_STATE), (7, D.DG_ERR_INVALID_ARG)):
        with pytest.raises(D.DGError) as e:
            h.profile_kernel(D.DG_PROF_APPLY, dt, 0, reps=2)
        assert e.value.status == st
    h.close()
