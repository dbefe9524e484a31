"""Checkpoint and resume of the residual loop.

The loop (``Space.residual_loop``, the device loop of dse_residual_loop)
chooses one descriptor per iteration; an interrupted search (a lost job, a
preempted node) would otherwise start again from r_0 = y.  Here the loop runs
one iteration per library call, resuming each call from the descriptors
chosen so far (dse_loop_desc.n_fixed / fixed: the fit with them and its
residual are recomputed on the device by the same refit kernels, so the
continued run takes the same bits as an uninterrupted one), and after every
iteration the state -- chosen ids, RMSEs, coefficients, the iteration's SIS
subspace and screen statistics -- is written to ``path`` atomically
(temporary file, fsync, rename), so a crash leaves either the previous or
the new checkpoint, never a partial one.

A checkpoint records a fingerprint of the problem (space size, sample
count, a hash of the target, k, precision); resuming against another
problem raises ValueError.  Host logic only: every iteration runs in the
CUDA library.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

FORMAT = 1


def fingerprint(space, y, k: int, precision: int) -> dict:
    """What a checkpoint must match to be resumed."""
    yb = np.ascontiguousarray(np.asarray(y, dtype=np.float64)).tobytes()
    return {"format": FORMAT, "n_stored": int(space.n_stored), "n_total": int(space.n_total),
            "n_samples": int(len(yb) // 8), "y_sha256": hashlib.sha256(yb).hexdigest(), "k": int(k),
            "precision": int(precision)}


def empty_state(fp: dict) -> dict:
    return {"fingerprint": fp, "chosen": [], "rmse": [], "coefs": [], "stats": [], "sis_ids": []}


def save(path: str, state: dict) -> None:
    """Atomic write: the file at ``path`` is either the old or the new state."""
    meta = {k: state[k] for k in ("fingerprint", "chosen", "rmse", "coefs", "stats")}
    sis = np.asarray(state["sis_ids"], dtype=np.uint64).reshape(len(state["sis_ids"]), -1)
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        np.savez(f, meta=np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8), sis_ids=sis)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def load(path: str):
    """The state in ``path``, or None when there is no checkpoint."""
    if not os.path.exists(path):
        return None
    with np.load(path) as z:
        meta = json.loads(bytes(z["meta"]).decode())
        sis = z["sis_ids"]
    meta["sis_ids"] = [row.copy() for row in sis]
    if len({len(meta[k]) for k in ("chosen", "rmse", "coefs", "stats", "sis_ids")}) != 1:
        raise ValueError(f"inconsistent checkpoint {path}")
    return meta


def residual_loop(space, y, n_iter: int, k: int, path: str, precision: int = 0, stop_after=None) -> dict:
    """The residual loop with a checkpoint after every iteration: resumes
    from ``path`` when it exists (same problem), runs the remaining
    iterations up to ``n_iter`` (or ``stop_after`` in total, to end a run
    early), and returns the state (chosen ids, RMSEs, coefficients, screen
    statistics and SIS subspaces of every iteration done)."""
    fp = fingerprint(space, y, k, precision)
    state = load(path)
    if state is None:
        state = empty_state(fp)
    elif state["fingerprint"] != fp:
        raise ValueError(f"checkpoint {path} belongs to another problem")
    end = n_iter if stop_after is None else min(n_iter, stop_after)
    for it in range(len(state["chosen"]), end):
        sis = np.full((it + 1) * k, np.iinfo(np.uint64).max, dtype=np.uint64)
        out = space.residual_loop(y, it + 1, k, precision=precision, sis_ids=sis, fixed=state["chosen"])
        if out["chosen"][:it] != state["chosen"]:
            raise RuntimeError("the library did not keep the fixed descriptors")
        state["chosen"].append(int(out["chosen"][it]))
        state["rmse"].append(float(out["rmse"][it]))
        state["coefs"].append([float(c) for c in out["coefs"][it]])
        state["stats"].append(out["stats"][it])
        state["sis_ids"].append(sis[it * k:(it + 1) * k].copy())
        save(path, state)
    return state
