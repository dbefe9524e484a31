"""Index-range sharding of one screen over several GPUs, one process per GPU.

The screened set is addressed by global candidate ids [0, n_total) (stored
features, then the flat indices of the last rung).  Each rank screens one
contiguous block of ids with ``Space.screen(id_begin=, id_end=)``; the only
exchange is one all-gather of every rank's per-list top-k (id, score, bound),
after which every rank merges them in the screen's own order (score
descending, id ascending).  The operands (stored rungs) are built on every
rank: they are small next to the candidate space.

Host logic only: the screening itself runs in the CUDA library on each rank.
"""
from __future__ import annotations

import numpy as np

_NO_ID = np.iinfo(np.uint64).max


def id_block(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous block [begin, end) of rank ``rank`` among ``world``: the
    first n_total % world ranks get one id more."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad partition")
    q, r = divmod(n_total, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def merge_topk(parts, k: int):
    """Merge (ids, scores, bounds) lists into the top k by (score desc, id
    asc).  Padding entries (id 2^64-1) are dropped."""
    ids = np.concatenate([np.asarray(p[0], np.uint64) for p in parts]) if parts else np.zeros(0, np.uint64)
    sc = np.concatenate([np.asarray(p[1], np.float64) for p in parts]) if parts else np.zeros(0)
    eb = np.concatenate([np.asarray(p[2], np.float64) for p in parts]) if parts else np.zeros(0)
    keep = ids != _NO_ID
    ids, sc, eb = ids[keep], sc[keep], eb[keep]
    order = np.lexsort((ids, -sc))[:k]
    return ids[order], sc[order], eb[order]


def gather_merge(lists, k: int, group=None):
    """All-gather every rank's lists [(ids, scores, bounds), ...] (same number
    of lists on every rank) and merge each list over the ranks."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    n_lists = len(lists)
    # fixed-size payload: k entries per list, padded
    pid = np.full((n_lists, k), _NO_ID, np.uint64)
    psc = np.full((n_lists, k), -np.inf)
    peb = np.zeros((n_lists, k))
    for l, (i, s, e) in enumerate(lists):
        m = min(k, len(i))
        pid[l, :m], psc[l, :m], peb[l, :m] = i[:m], s[:m], e[:m]
    payload = np.concatenate([pid.view(np.float64), psc, peb], axis=1)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.from_numpy(payload).to(dev)
    out = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    got = [o.cpu().numpy() for o in out]
    merged = []
    for l in range(n_lists):
        parts = []
        for g in got:
            parts.append((g[l, :k].copy().view(np.uint64), g[l, k:2 * k], g[l, 2 * k:]))
        merged.append(merge_topk(parts, k))
    return merged


def sharded_screen(space, Y, k: int, group=None, **screen_kw):
    """Screen the whole space of ``space`` over the ranks of ``group``: this
    rank's id block on its own GPU, then the all-gather merge.  Returns the
    merged lists and this rank's statistics."""
    import torch.distributed as dist

    world, rank = dist.get_world_size(group), dist.get_rank(group)
    b, e = id_block(space.n_total, world, rank)
    if e == b:  # more ranks than candidates: nothing to screen here (id_end 0 would mean "all")
        T = 1 if Y.ndim == 1 else Y.shape[0]
        n_lists = 1 if screen_kw.get("mode", 0) == 1 else T
        empty = (np.zeros(0, np.uint64), np.zeros(0), np.zeros(0))
        return gather_merge([empty] * n_lists, k, group), None
    res = space.screen(Y, k, id_begin=b, id_end=e, **screen_kw)
    lists = [res.fetch(l) for l in range(res.n_lists)]
    stats = res.stats()
    res.free()
    return gather_merge(lists, k, group), stats
