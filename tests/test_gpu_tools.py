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


@pytest.mark.parametrize("kernel", ["dots", "update", "apply32", "assemble"])
def test_profile_case_kernels(kernel):
    out = _run("paper_1502_02941_gb300.profile_case", "--kernel", kernel, "--N", "32", "--reps", "2")
    assert out["ms"] > 0
