"""GPU parity of the batched screen (dse_sis_screen_batched): many problems,
each a space built on a sample gather list of its base data set (cross-
validation folds and bootstrap resamples) with its own target, k per problem.

  * small batch (32 problems, N <= 300): every problem against the oracle run
    on that problem alone -- reason counts bit-exact, top-k equal apart from
    ties, scores within 1e-5 relative and within the reported bound;
  * the full 256-problem workload: a spread of problems equal (ids, scores)
    to the single-problem screen of the same space, every returned entry
    re-scored by the oracle; a CUDA-graph re-screen with new targets equal to
    an eager batch with those targets.
"""
import numpy as np
import pytest

import __graft_entry__ as ge

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ge.build()
    import oracle
    from paper_2602_06986_gb300 import dse
    from paper_2602_06986_gb300 import workloads as W

    return torch, oracle, dse, W


def _build(env, w):
    torch, oracle, dse, W = env
    kw = dict(unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    Xd = [torch.from_numpy(b["X"]).cuda() for b in w["bases"]]
    spaces, targets = [], []
    for p in w["problems"]:
        b = w["bases"][p["base"]]
        spaces.append(dse.Space(Xd[p["base"]], b["units"], w["op_mask"], w["max_rung"], sample_idx=p["samples"],
                                **kw))
        targets.append(b["y"][p["samples"]])
    return spaces, targets


def _oracle_space(env, w, p):
    torch, oracle, dse, W = env
    b = w["bases"][p["base"]]
    return oracle.Space(np.ascontiguousarray(b["X"][:, p["samples"]]), b["units"], w["op_mask"], w["max_rung"],
                        unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])


def _same_topk(a, b, tol=TOL):
    """Two exact top-k lists of the same problem: rank-wise scores within tol
    (each side may report an FP32 or an FP64 re-scored value) and equal sets
    apart from candidates tied with the k-th score."""
    (ia, sa, _), (ib, sb, _) = a, b
    assert len(ia) == len(ib)
    np.testing.assert_allclose(sa, sb, rtol=tol, atol=1e-12)
    sk = min(sa[-1], sb[-1])
    score = dict(zip(ia.tolist(), sa.tolist()))
    score.update(zip(ib.tolist(), sb.tolist()))
    for x in set(ia.tolist()) ^ set(ib.tolist()):
        assert abs(score[x] - sk) <= tol * sk + 1e-12, x


def test_small_batch_matches_oracle(env):
    torch, oracle, dse, W = env
    w = W.batched(1, n_base=4, n_hi=300, p_hi=12)
    spaces, targets = _build(env, w)
    k = w["k"]
    bt = dse.Batch(spaces, targets, k)
    for i, p in enumerate(w["problems"]):
        orc = _oracle_space(env, w, p)
        assert spaces[i].n_stored == orc.n_features
        y = targets[i][None, :]
        oids, osc, ocnt = orc.screen(y, k)
        st = bt.stats(i)
        assert st["reasons"] == ocnt, i
        assert st["screened"] == orc.total_candidates
        ids, sc, eb = bt.fetch(i)
        ge._check_topk(ids, sc, eb, oids[0], osc[0], orc, y, 0, tol=TOL)
    bt.free()


def test_small_batch_fp64(env):
    torch, oracle, dse, W = env
    w = W.batched(2, n_base=2, n_hi=200, p_hi=11)
    spaces, targets = _build(env, w)
    k = 50
    bt = dse.Batch(spaces, targets, k, precision=dse.PREC_FP64)
    for i, p in enumerate(w["problems"]):
        orc = _oracle_space(env, w, p)
        y = targets[i][None, :]
        oids, osc, ocnt = orc.screen(y, k)
        assert bt.stats(i)["reasons"] == ocnt, i
        ids, sc, eb = bt.fetch(i)
        ge._check_topk(ids, sc, eb, oids[0], osc[0], orc, y, 0, tol=TOL)


def test_full_batch_against_single_and_oracle(env):
    torch, oracle, dse, W = env
    w = W.batched(0)
    assert len(w["problems"]) == 256
    spaces, targets = _build(env, w)
    k = w["k"]
    bt = dse.Batch(spaces, targets, k, graph=True)
    res = [bt.fetch(i) for i in range(len(spaces))]
    stats = [bt.stats(i) for i in range(len(spaces))]
    for i, sp in enumerate(spaces):
        assert stats[i]["screened"] == sp.n_total
        assert sum(stats[i]["reasons"].values()) == sp.n_total
        assert len(res[i][0]) == k
    # a spread of problems (smallest and largest bases, folds and bootstraps)
    for i in [0, 5, 7, 8, 12, 15, 100, 255]:
        r = spaces[i].screen(torch.from_numpy(targets[i]).cuda(), k)
        assert r.stats()["reasons"] == stats[i]["reasons"], i
        _same_topk(r.fetch(0), res[i])
    # every returned entry re-scored by the oracle (FP64), in order
    for i, p in enumerate(w["problems"]):
        if i % 4:
            continue
        orc = _oracle_space(env, w, p)
        ids, sc, eb = res[i]
        ref, why = orc.score_ids(targets[i][None, :], ids)
        assert np.all(why == 0), i
        err = np.abs(sc - ref[:, 0])
        assert np.all(err <= TOL * ref[:, 0] + 1e-12), i
        assert np.all(err <= eb + 1e-12), i
        assert np.all(np.diff(sc) <= 0), i
    # graph re-screen with new targets == an eager batch with those targets
    rng = np.random.default_rng(5)
    new = [t[rng.permutation(len(t))] + 0.1 * t for t in targets]
    bt.rescreen(np.concatenate(new))
    bt.rescreen(np.concatenate(new))  # second replay of the captured graph
    eager = dse.Batch(spaces, new, k)
    for i in range(0, len(spaces), 17):
        _same_topk(bt.fetch(i), eager.fetch(i))
        assert bt.stats(i)["reasons"] == eager.stats(i)["reasons"]
    bt.free()
    eager.free()
