"""Training and evaluation driver of the learned preconditioner on batches of
the learned workload (64x64 split squares, P2, batched-workload coefficients).

Training residuals come from the method's own f64 block-Jacobi GMRES solves of
the training batch: r = F - A x_k for the iterates x_k after k steps, and the
Krylov basis vectors of those solves (the vectors the preconditioner is applied
to inside GMRES); each is paired (inside the library) with its one-layer-overlap
patch correction.
"""
from __future__ import annotations

import json
import struct
import time

import numpy as np

from . import dg as D
from . import problem
from . import workloads as W

TRAIN_FAMILY = "learned"


def make_batch(h: D.DG, n_inst: int, N: int, first: int = 0, k: int = 2, store=D.DG_STORE_F64, **params):
    """Instances first .. first+n_inst-1 of the learned workload's draw."""
    cfgs, i = [], first
    while len(cfgs) < n_inst:
        c = W.random_instance(TRAIN_FAMILY, i, N_fixed=N, k_fixed=k)
        i += 1
        cfgs.append(c)
    ma, starts = W.concat_meshes([W.structured_mesh(c.N) for c in cfgs])
    coeffs = np.array([[c.problem.eps, c.problem.alpha, *c.problem.b] for c in cfgs])
    problem.setup_batch(h, cfgs, ma, starts, coeffs, store=store, **params)
    h.precond_setup()
    return cfgs, ma, starts


def collect(h: D.DG, snapshots=(10, 30, 60, 100, 200, 400), basis_at=(40, 90, 240), nvec=30, tol=1e-10,
            max_it=20000):
    """Solve the current batch with block-Jacobi GMRES and record one training
    row per element for the zero iterate and each snapshot iterate, and for
    the first nvec Krylov basis vectors of the restart cycle running after
    each count in basis_at."""
    h.set_params(precond=D.DG_PRECOND_BLOCK_JACOBI, tol=tol, max_it=max_it)
    xstar, its, rr, st = h.batch_solve(D.DG_F64, raise_on_nonconv=False)
    h.mlp_collect(h.torch.zeros_like(xstar))
    for k in snapshots:
        h.set_params(max_it=k)
        xk, _, _, _ = h.batch_solve(D.DG_F64, raise_on_nonconv=False)
        h.mlp_collect(xk)
    for k in basis_at:
        h.set_params(max_it=k)
        h.batch_solve(D.DG_F64, raise_on_nonconv=False)
        h.mlp_collect_basis(min(nvec, h.params.gmres_m + 1))
    h.set_params(max_it=max_it)
    return its, rr, st


SCHEDULE = ((1e-3, 0.5), (3e-4, 0.3), (1e-4, 0.2))   # (learning rate, share of the steps)


def train(h: D.DG, steps=12000, batch_rows=8192, seed=0, schedule=SCHEDULE):
    """Adam over the collected rows with a stepwise learning-rate decay."""
    t0 = time.perf_counter()
    losses = []
    for i, (lr, share) in enumerate(schedule):
        n = max(1, int(round(steps * share)))
        losses.append(h.mlp_train(n, batch_rows=batch_rows, lr=lr, seed=seed + 7919 * i))
    return np.concatenate(losses), time.perf_counter() - t0


def evaluate(h: D.DG, max_it=20000, tol=1e-10):
    """Batched f64 solves of the current batch with block Jacobi and with the
    learned preconditioner: per-instance iterations, relres, wall time."""
    import torch
    out = {}
    for name, pc in (("bj", D.DG_PRECOND_BLOCK_JACOBI), ("mlp", D.DG_PRECOND_MLP)):
        h.set_params(precond=pc, tol=tol, max_it=max_it)
        h.batch_solve(D.DG_F64, raise_on_nonconv=False)          # warm-up (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, its, rr, st = h.batch_solve(D.DG_F64, raise_on_nonconv=False)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "its": its.copy(), "relres": rr.copy(),
                     "converged": int((st == 0).sum())}
    h.set_params(precond=D.DG_PRECOND_BLOCK_JACOBI)
    return out


# ---------------------------------------------------------------------------
# checkpoints of the trained network
# ---------------------------------------------------------------------------
# File layout (little-endian): 8-byte magic b"DGMLPW1\0", uint32 header length
# L, L bytes of UTF-8 JSON {"degree", "n_params", "dtype": "float32", "seed",
# "config"}, then n_params float32 values (the flat vector of
# dg_mlp_set_weights / dg_mlp_get_weights).
_MAGIC = b"DGMLPW1\0"


def save_weights(path, theta, degree: int, seed: int = 0, config: dict | None = None) -> None:
    """Write the network's flat parameter vector with a header (degree, size,
    training seed and settings) to a file path or a binary file object."""
    theta = np.ascontiguousarray(theta, dtype="<f4").reshape(-1)
    n = D.dg_mlp_num_params(degree)
    if theta.size != n:
        raise ValueError(f"{theta.size} parameters given, degree {degree} has {n}")
    head = json.dumps({"degree": int(degree), "n_params": int(n), "dtype": "float32", "seed": int(seed),
                       "config": config or {}}, sort_keys=True).encode()
    blob = _MAGIC + struct.pack("<I", len(head)) + head + theta.tobytes()
    if hasattr(path, "write"):
        path.write(blob)
    else:
        with open(path, "wb") as fh:
            fh.write(blob)


def load_weights(path):
    """Read a checkpoint written by save_weights (a file path or a binary file
    object); returns (theta float32, header).  Raises ValueError for a foreign
    or truncated file or a size that does not match the degree."""
    if hasattr(path, "read"):
        data = path.read()
    else:
        with open(path, "rb") as fh:
            data = fh.read()
    if len(data) < 12 or data[:8] != _MAGIC:
        raise ValueError("not a network checkpoint")
    (hl,) = struct.unpack("<I", data[8:12])
    if len(data) < 12 + hl:
        raise ValueError("truncated header")
    try:
        head = json.loads(data[12:12 + hl].decode())
    except (UnicodeDecodeError, ValueError) as e:
        raise ValueError(f"unreadable checkpoint header: {e}") from None
    if not isinstance(head, dict):
        raise ValueError("checkpoint header is not a JSON object")
    deg = head.get("degree")
    if not isinstance(deg, int) or isinstance(deg, bool) or not 1 <= deg <= 3:
        raise ValueError(f"checkpoint header has no valid degree (1..3): {deg!r}")
    n = D.dg_mlp_num_params(deg)
    if head.get("dtype") != "float32" or head.get("n_params") != n or len(data) != 12 + hl + 4 * n:
        raise ValueError("checkpoint size does not match its degree")
    theta = np.frombuffer(data, dtype="<f4", count=n, offset=12 + hl).astype(np.float32)
    return theta, head
