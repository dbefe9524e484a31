"""Host logic of the multi-GPU index-range sharding, on CPU: id blocks cover
the space exactly, the top-k merge keeps the screen's order, and a
world_size-2 gloo run (each rank screening its block with the oracle in place
of its GPU) merges to the oracle's full screen."""
import os
import socket

import numpy as np
import pytest

from paper_2602_06986_gb300 import shard


def test_id_blocks_partition():
    for n in [0, 1, 7, 100, 2 ** 40 + 3]:
        for world in [1, 2, 3, 8]:
            blocks = [shard.id_block(n, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            for (a, b), (c, d) in zip(blocks, blocks[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.id_block(10, 2, 2)


def test_merge_order_and_ties():
    a = (np.array([5, 9, 2], np.uint64), np.array([0.9, 0.5, 0.5]), np.array([1e-7, 1e-7, 1e-7]))
    b = (np.array([1, 3, 2 ** 64 - 1], np.uint64), np.array([0.5, 0.95, -np.inf]), np.zeros(3))
    ids, sc, eb = shard.merge_topk([a, b], 4)
    assert ids.tolist() == [3, 5, 1, 2]  # equal scores: lower id first
    assert sc.tolist() == [0.95, 0.9, 0.5, 0.5]
    ids, _, _ = shard.merge_topk([a, b], 10)
    assert len(ids) == 5  # padding dropped


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    from paper_2602_06986_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = W.tiny(4)
        orc = oracle.Space(w["X"], w["units"], w["op_mask"], w["max_rung"])
        rng = np.random.default_rng(9)
        Y = np.stack([w["Y"][0], w["X"][2] * w["X"][5] + 0.05 * rng.standard_normal(w["X"].shape[1])])
        k = 40
        b, e = shard.id_block(orc.total_candidates, world, rank)
        ids, sc, cnt = orc.screen(Y, k, id_begin=b, id_end=e)
        lists = [(ids[l], sc[l], np.zeros(len(ids[l]))) for l in range(2)]
        merged = shard.gather_merge(lists, k)
        if rank == 0:
            fids, fsc, _ = orc.screen(Y, k)
            ok = all(np.array_equal(merged[l][0], fids[l]) and np.array_equal(merged[l][1], fsc[l])
                     for l in range(2))
            q.put(ok)
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_merge_equals_full_screen():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get() is True
