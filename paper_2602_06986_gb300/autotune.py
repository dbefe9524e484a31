"""Autotuner of the planner's launch and tile parameters.

The library's planner has a few parameters that decide how the work of a
screen is cut and ordered, not what is computed (dse_set_tuning): the number
of i-blocks per group of pair tiles (which tiles run side by side and share
operand rows in L2), the stride of the seed tiles launched first, the largest
N for the product Gram contraction, the number of targets from which the
tensor cores are used, the work per job of a batched screen, and the
a-blocks per group of the multi-target Gram kernel's tile order.  This module
times candidate values on the device for a workload class and keeps the
fastest in a JSON cache keyed by (kernel, N bucket, T bucket); ``apply``
installs the cached choice before a screen of that class.

The search is coordinate descent from the defaults: one parameter at a time
over its candidate values, the others held at the best so far, each setting
timed ``reps`` times (median); a value replaces the current one only when it
is faster by more than ``margin`` (relative), so noise does not move the
choice.  Host logic only: the screens themselves run in the CUDA library.
"""
from __future__ import annotations

import json
import math
import os
import statistics

# candidate values per tuned kernel class
CANDIDATES = {
    # tensor-core multi-target screen (product/quotient tiles)
    "screen_tc": {"tile_group": [2, 4, 8, 16], "seed_stride": [32, 64, 128]},
    # multi-target Gram screen: a-blocks per group of its tile order, and
    # whether 2..16 targets take it (8) or the CUDA-core kernels (17)
    "screen_gmt": {"gmt_group": [1, 5, 4096], "gmt_cluster": [1], "tc_min_targets": [8, 17]},
    # CUDA-core screens (one target, or sample by sample)
    "screen_cc": {"tile_group": [1, 2, 4, 8]},
    # one target with 16 <= N <= 2048: Gram contraction (2048) or direct (16)
    "screen_single": {"gram_max_n": [16, 2048]},
    # batched screens of many small problems
    "batched": {"batch_job_samples": [4096, 8192, 16384, 32768, 65536]},
}


def bucket_n(N: int) -> int:
    """Power-of-two bucket of the sample count."""
    if N < 1:
        raise ValueError("N must be positive")
    return 1 << max(0, math.ceil(math.log2(N)))


def bucket_t(T: int) -> str:
    """Target-count class: 1, 2-7, 8-16, 17-32, 33-64, >64."""
    if T < 1:
        raise ValueError("T must be positive")
    for hi, name in ((1, "1"), (7, "2-7"), (16, "8-16"), (32, "17-32"), (64, "33-64")):
        if T <= hi:
            return name
    return ">64"


def key(kernel: str, N: int, T: int) -> str:
    return f"{kernel}|N{bucket_n(N)}|T{bucket_t(T)}"


def cuda_timer(fn) -> float:
    """Seconds one call of fn takes on the current CUDA stream (events, after
    a synchronisation on both sides)."""
    import torch

    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def tune(kernel: str, N: int, T: int, run, cache: dict | None = None, timer=None, reps: int = 3,
         margin: float = 0.02, install=None, candidates: dict | None = None, warmup: int = 1) -> dict:
    """Tune ``kernel`` for the class of (N, T).  ``run()`` executes the
    workload once under the installed settings; ``install(config)`` installs
    a settings dict (default: dse.set_tuning).  ``warmup`` untimed runs under
    the defaults come first (the first runs of a process load modules and
    allocate, which would bias the defaults' timing).  Returns the cache
    entry {"config", "seconds", "tried"}; with a cache that already holds the
    key, returns it without timing or running anything."""
    cache = {} if cache is None else cache
    k = key(kernel, N, T)
    if k in cache:
        return cache[k]
    if timer is None:
        timer = cuda_timer
    if install is None:
        from . import dse

        install = dse.set_tuning
    grid = (candidates or CANDIDATES)[kernel]
    tried = []

    def measure(cfg):
        install(cfg)
        t = statistics.median(timer(run) for _ in range(reps))
        tried.append({"config": dict(cfg), "seconds": t})
        return t

    try:
        install({})
        for _ in range(warmup):
            run()
        best = {}  # empty: every default
        t_best = measure(best)
        for name, values in grid.items():
            for v in values:
                cfg = dict(best, **{name: v})
                if cfg == best:
                    continue
                t = measure(cfg)
                if t < t_best * (1.0 - margin):
                    best, t_best = cfg, t
    finally:
        install(None)
    entry = {"config": best, "seconds": t_best, "tried": tried}
    cache[k] = entry
    return entry


def lookup(cache: dict, kernel: str, N: int, T: int):
    """The cached settings for the class of (N, T), or None."""
    e = cache.get(key(kernel, N, T))
    return None if e is None else dict(e["config"])


def apply(cache: dict, kernel: str, N: int, T: int, install=None) -> dict | None:
    """Install the cached settings for the class (the defaults if none)."""
    if install is None:
        from . import dse

        install = dse.set_tuning
    cfg = lookup(cache, kernel, N, T)
    install(cfg if cfg else None)
    return cfg


def load(path: str) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def save(path: str, cache: dict) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
