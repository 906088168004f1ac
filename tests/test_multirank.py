"""Multi-rank host logic of the benchmark on CPU: world_size-2 gloo ranks.

The solve path does not shard (replicas only): each rank solves its own
copy of the workload, and the only collectives are the barrier and the
max-over-ranks timing.  These tests run that timing logic and the
reference arm's rank handling on gloo, without a GPU."""
import io
import contextlib
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 100.0 + 50.0 * rank          # rank 1 is the slower one
        ms = bench.max_over_ranks(ms_local, world)
        value = bench.whole_job_value(2 * 3, world, ms)   # 2 solves x 3 steps per rank
        # the reference arm: rank 0 alone runs and prints; other ranks return at once
        buf = io.StringIO()
        if rank != 0:
            with contextlib.redirect_stdout(buf):
                bench.reference_arm(None, rank)
        dist.barrier()
        out[rank] = (ms, value, buf.getvalue())
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_on_two_gloo_ranks():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    for rank in range(world):
        ms, value, printed = res[rank]
        assert ms == 150.0                       # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 3 * world / 0.150)
        assert printed == ""                     # no reference line from rank 1 (nor work)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(123.0, 1) == 123.0
    assert bench.whole_job_value(2, 1, 500.0) == pytest.approx(4.0)


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference (the oracle on the host cores) prints one JSON
    line with the contract's keys, on the same metric and workload as the GPU
    arm."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["value"] > 0
    assert d["config"]["workload"] == bench.WORKLOAD and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_batched_workload_grouped_by_degree_keeps_each_draw():
    """The bench's batched workload: instances 0..63 of the batched family,
    one batch per drawn degree; every instance keeps its own seeded draw."""
    from paper_1502_02941_gb300 import workloads as W
    groups = W.batch_by_degree("batched", 64)
    assert sorted(groups) == [1, 2] and sum(len(g[0]) for g in groups.values()) == 64
    for k, (cfgs, ma, starts, coeffs) in groups.items():
        assert all(c.k == k for c in cfgs)
        assert starts[-1] == ma.elems.shape[0] == sum(2 * c.N ** 2 for c in cfgs)
        for c, row in zip(cfgs, coeffs):
            i = int(c.name.split("inst")[1])
            d = W.random_instance("batched", i)
            assert (d.N, d.k, d.problem.eps, d.problem.alpha) == (c.N, c.k, row[0], row[1])
