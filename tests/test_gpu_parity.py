"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Bars (scores relative 1e-5 is the stated tolerance of the method's FP32 path):
  * counts per rung and per reason, stored-feature count, candidate count,
    expression strings and returned ids: bit-exact;
  * every returned score within 1e-5 relative of the oracle's FP64 score and
    within the bound the library reports with it;
  * top-k sets equal apart from candidates whose oracle score lies within
    1e-5 * s_k of the k-th oracle score s_k (interchangeable ties).
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


def spaces(env, w, **extra):
    torch, oracle, dse, W = env
    kw = dict(unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    kw.update(extra)
    sp = dse.Space(torch.from_numpy(w["X"]).cuda(), w["units"], w["op_mask"], w["max_rung"], **kw)
    orc = oracle.Space(w["X"], w["units"], w["op_mask"], w["max_rung"], **kw)
    return sp, orc


def check_counts(sp, orc, max_rung):
    assert sp.n_stored == orc.n_features
    assert sp.n_total == orc.total_candidates
    for r in range(max_rung):
        assert sp.counts(r) == orc.rung_counts(r), r


def check_list(ids, sc, eb, oids, osc, orc, Y, t):
    ge._check_topk(ids, sc, eb, oids, osc, orc, Y, t, tol=TOL)


def assert_same_topk(ids_m, sc_m, eb_m, ids_f, sc_f, eb_f):
    """Two top-k lists of one screen taken different ways (merged range
    screens and the full screen) agree up to ties inside the scores' bounds
    (the method's parity target is top-k sets identical apart from ties
    inside the score tolerance, 1e-5 relative):
    a candidate's reported score may come from the FP32 or the FP32-pair
    re-score depending on how it was classified in its own screen, so
    members whose scores lie within the bounds of the k-th score are
    interchangeable; every member clear of that band is in both lists, and
    common members' scores agree within their bounds."""
    assert len(ids_m) == len(ids_f)
    if len(ids_f) == 0:
        return
    band = 2.0 * (float(np.max(eb_m)) + float(np.max(eb_f))) + 1e-12
    kth = max(float(sc_m[-1]), float(sc_f[-1]))
    sm, sf = set(int(i) for i in ids_m), set(int(i) for i in ids_f)
    assert {int(i) for i, s in zip(ids_m, sc_m) if s > kth + band} <= sf
    assert {int(i) for i, s in zip(ids_f, sc_f) if s > kth + band} <= sm
    fm = {int(i): (s, e) for i, s, e in zip(ids_m, sc_m, eb_m)}
    for i, s, e in zip(ids_f, sc_f, eb_f):
        if int(i) in fm:
            s2, e2 = fm[int(i)]
            assert abs(s - s2) <= e + e2 + 1e-12, (int(i), s, s2)
    assert len(sm & sf) >= len(ids_f) - sum(1 for s in sc_f if s <= kth + band)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_parity(env, seed):
    torch, oracle, dse, W = env
    w = W.tiny(seed)
    sp, orc = spaces(env, w)
    check_counts(sp, orc, w["max_rung"])
    res = sp.screen(torch.from_numpy(w["Y"]).cuda(), w["k"])
    ids, sc, eb = res.fetch(0)
    oids, osc, ocnt = orc.screen(w["Y"], w["k"])
    check_list(ids, sc, eb, oids[0], osc[0], orc, w["Y"], 0)
    st = res.stats()
    assert st["reasons"] == ocnt
    assert [sp.expr(int(i)) for i in ids] == [orc.expr(int(i)) for i in ids]
    # a-priori counts of the streamed rung
    slots, rs = sp.counts(w["max_rung"])
    oslots, ors = orc.rung_counts(w["max_rung"])
    assert slots == oslots
    for key in ("unit", "complexity", "domain", "magnitude"):
        assert rs[key] == ors[key], key
    assert rs["valid"] == ors["valid"] + ors["realised"]


@pytest.mark.parametrize("direct", [False, True])
def test_medium_parity(env, direct):
    """Products and quotients from the tensor-core Gram contraction (default
    for one FP32 target) and sample by sample (DSE_FLAG_DIRECT)."""
    torch, oracle, dse, W = env
    w = W.medium(0)
    sp, orc = spaces(env, w)
    check_counts(sp, orc, w["max_rung"])
    res = sp.screen(torch.from_numpy(w["Y"]).cuda(), w["k"], flags=dse.FLAG_DIRECT if direct else 0)
    ids, sc, eb = res.fetch(0)
    oids, osc, ocnt = orc.screen(w["Y"], w["k"])
    check_list(ids, sc, eb, oids[0], osc[0], orc, w["Y"], 0)
    st = res.stats()
    assert st["reasons"] == ocnt
    assert st["valid_by_group"][1] > 0


@pytest.mark.parametrize("seed", [0, 3])
def test_fp64_plain_parity(env, seed):
    torch, oracle, dse, W = env
    w = W.tiny(seed)
    sp, orc = spaces(env, w)
    res = sp.screen(torch.from_numpy(w["Y"]).cuda(), w["k"], precision=dse.PREC_FP64)
    ids, sc, eb = res.fetch(0)
    oids, osc, ocnt = orc.screen(w["Y"], w["k"])
    check_list(ids, sc, eb, oids[0], osc[0], orc, w["Y"], 0)
    ref, _ = orc.score_ids(w["Y"], ids)
    assert np.max(np.abs(sc - ref[:, 0]) / ref[:, 0]) < 1e-12
    assert res.stats()["reasons"] == ocnt


@pytest.mark.parametrize("T,mode", [(3, "per_target"), (5, "aggregated"), (17, "per_target")])
def test_multi_target(env, T, mode):
    torch, oracle, dse, W = env
    w = W.tiny(4)
    rng = np.random.default_rng(9)
    X = w["X"]
    Y = np.stack([X[rng.integers(8)] * X[rng.integers(8)] / X[rng.integers(8)] + 0.05 * rng.standard_normal(100)
                  for _ in range(T)])
    sp, orc = spaces(env, w)
    m = dse.MODE_AGGREGATED if mode == "aggregated" else dse.MODE_PER_TARGET
    k = 60
    res = sp.screen(torch.from_numpy(Y).cuda(), k, mode=m)
    oids, osc, ocnt = orc.screen(Y, k, mode=mode)
    lists = 1 if mode == "aggregated" else T
    for l in range(lists):
        ids, sc, eb = res.fetch(l)
        if mode == "aggregated":
            ref, _ = orc.score_ids(Y, ids)
            agg = np.sqrt(np.mean(ref ** 2, axis=1))
            assert np.all(np.abs(sc - agg) <= TOL * agg)
            sk = osc[0][-1]
            above = {int(i) for i, s in zip(oids[0], osc[0]) if s > sk * (1 + TOL)}
            assert above <= {int(i) for i in ids}
        else:
            check_list(ids, sc, eb, oids[l], osc[l], orc, Y, l)
    assert res.stats()["reasons"] == ocnt


@pytest.mark.parametrize("wname,T,flags", [("tiny", 17, 0), ("tiny", 40, 0), ("medium", 8, 4), ("medium", 33, 0),
                                           ("tiny", 3, 0), ("tiny", 16, 0), ("medium", 8, 0), ("medium", 16, 0)])
def test_tensor_core_multi_target(env, wname, T, flags):
    """BF16x3 tcgen05 contractions against the oracle, per target: the
    sample-by-sample kernel (one TMEM block at N=100, drained blocks at
    N=1000; above 16 targets, or with DSE_FLAG_DIRECT) and the multi-target
    Gram kernel (2..16 targets)."""
    torch, oracle, dse, W = env
    w = getattr(W, wname)(7)
    X = w["X"]
    rng = np.random.default_rng(T)
    N = X.shape[1]
    Y = np.stack([X[rng.integers(len(X))] * X[rng.integers(len(X))] / X[rng.integers(len(X))]
                  + 0.05 * rng.standard_normal(N) for _ in range(T)])
    sp, orc = spaces(env, w)
    k = 50
    res = sp.screen(torch.from_numpy(Y).cuda(), k, precision=dse.PREC_BF16X3, flags=flags)
    st = res.stats()
    assert st["precision_used"] == dse.PREC_BF16X3
    assert st["binary_path"] == (dse.PATH_GRAM_MT if T <= 16 and not flags else dse.PATH_TENSOR)
    oids, osc, ocnt = orc.screen(Y, k)
    assert st["reasons"] == ocnt
    for l in range(T):
        ids, sc, eb = res.fetch(l)
        check_list(ids, sc, eb, oids[l], osc[l], orc, Y, l)


def test_ranges_merge_to_full(env):
    """Screening disjoint ragged id ranges and merging their top-k equals the
    full screen (the index-range sharding of the multi-GPU plan)."""
    torch, oracle, dse, W = env
    w = W.tiny(5)
    sp, orc = spaces(env, w)
    Yd = torch.from_numpy(w["Y"]).cuda()
    full = sp.screen(Yd, 50).fetch(0)
    cuts = [0, 37, 1000, 7777, 20011, sp.n_total]
    parts = []
    counts = {}
    for a, b in zip(cuts[:-1], cuts[1:]):
        r = sp.screen(Yd, 50, id_begin=a, id_end=b)
        parts.append(r.fetch(0))
        st = r.stats()
        assert st["screened"] == b - a
        for kk, v in st["reasons"].items():
            counts[kk] = counts.get(kk, 0) + v
        oi, os_, oc = orc.screen(w["Y"], 50, id_begin=a, id_end=b)
        assert st["reasons"] == oc
    ids = np.concatenate([p[0] for p in parts])
    sc = np.concatenate([p[1] for p in parts])
    eb = np.concatenate([p[2] for p in parts])
    order = np.lexsort((ids, -sc))[:50]
    assert_same_topk(ids[order], sc[order], eb[order], *full)


def test_gram_multi_target_ranges_and_edges(env):
    """Multi-target Gram path (4 targets): disjoint ragged id ranges (one of
    a single binary candidate, one empty) merge to the full screen list by
    list with the oracle's counts; k = 1 and k above the valid count."""
    torch, oracle, dse, W = env
    w = W.tiny(5)
    sp, orc = spaces(env, w)
    rng = np.random.default_rng(4)
    N = w["X"].shape[1]
    Y = np.stack([w["Y"][0] + 0.2 * rng.standard_normal(N) for _ in range(4)])
    Yd = torch.from_numpy(Y).cuda()
    full = sp.screen(Yd, 40, precision=dse.PREC_BF16X3)
    assert full.stats()["binary_path"] == dse.PATH_GRAM_MT
    b0 = sp.n_stored + 6 * 100  # inside the binary block of the tiny space
    cuts = [0, 37, b0, b0 + 1, b0 + 1, 7777, 20011, sp.n_total]
    parts = [[] for _ in range(4)]
    for a, b in zip(cuts[:-1], cuts[1:]):
        r = sp.screen(Yd, 40, id_begin=a, id_end=b, precision=dse.PREC_BF16X3)
        st = r.stats()
        assert st["screened"] == b - a
        oi, os_, oc = orc.screen(Y, 40, id_begin=a, id_end=b)
        assert st["reasons"] == oc, (a, b)
        for l in range(4):
            parts[l].append(r.fetch(l))
            check_list(*parts[l][-1], oi[l], os_[l], orc, Y, l)
    for l in range(4):
        ids = np.concatenate([p[0] for p in parts[l]])
        sc = np.concatenate([p[1] for p in parts[l]])
        eb = np.concatenate([p[2] for p in parts[l]])
        order = np.lexsort((ids, -sc))[:40]
        assert_same_topk(ids[order], sc[order], eb[order], *full.fetch(l))
    # k = 1 and k above the number of valid candidates
    r = sp.screen(Yd, 1, precision=dse.PREC_BF16X3)
    oi, os_, oc = orc.screen(Y, 1)
    for l in range(4):
        ids, sc, eb = r.fetch(l)
        assert abs(sc[0] - os_[l][0]) <= TOL * os_[l][0]
    r = sp.screen(Yd, 10 ** 6, id_begin=b0, id_end=b0 + 3000, precision=dse.PREC_BF16X3)
    oi, os_, oc = orc.screen(Y, 10 ** 6, id_begin=b0, id_end=b0 + 3000)
    for l in range(4):
        ids, sc, eb = r.fetch(l)
        assert len(ids) == oc["valid"] == len(oi[l])
        check_list(ids, sc, eb, oi[l], os_[l], orc, Y, l)


def test_edge_cases(env):
    torch, oracle, dse, W = env
    w = W.tiny(6)
    sp, orc = spaces(env, w)
    Yd = torch.from_numpy(w["Y"]).cuda()
    # k larger than the number of valid candidates: everything, sorted
    r = sp.screen(Yd, 10 ** 6, id_begin=0, id_end=300)
    ids, sc, eb = r.fetch(0)
    oi, os_, oc = orc.screen(w["Y"], 10 ** 6, id_begin=0, id_end=300)
    assert len(ids) == oc["valid"] == len(oi[0])
    check_list(ids, sc, eb, oi[0], os_[0], orc, w["Y"], 0)
    # k = 1
    ids, sc, eb = sp.screen(Yd, 1).fetch(0)
    oi, os_, _ = orc.screen(w["Y"], 1)
    assert abs(sc[0] - os_[0][0]) <= TOL * os_[0][0]
    # empty range
    ids, sc, eb = sp.screen(Yd, 5, id_begin=100, id_end=100).fetch(0)
    assert len(ids) == 0
    # range past the end
    with pytest.raises(dse.DseError) as e:
        sp.screen(Yd, 5, id_begin=0, id_end=sp.n_total + 1)
    assert e.value.status == dse.ERANGE
    # constant target
    with pytest.raises(dse.DseError) as e:
        sp.screen(torch.ones(1, 100, dtype=torch.float64, device="cuda"), 5).fetch(0)
    assert e.value.status == dse.EINVAL
    # decode past the end
    with pytest.raises(dse.DseError) as e:
        sp.decode(sp.n_total)
    assert e.value.status == dse.ERANGE


def test_tiny_samples_and_degenerate_primary(env):
    """N = 3 samples, a constant primary (dropped by the realised test), ops
    that trip every domain rule."""
    torch, oracle, dse, W = env
    X = np.array([[0.5, 1.5, 2.5], [2.0, 2.0, 2.0], [-1.0, 0.25, 3.0], [1.0, 2.0, 4.0]])
    units = np.array([[1], [0], [1], [0]], np.int32)
    y = np.array([1.0, 3.0, 2.0])
    for ops in (W.OPS_FULL, W.OPS_TINY):
        sp = dse.Space(torch.from_numpy(X).cuda(), units, ops, 2)
        orc = oracle.Space(X, units, ops, 2)
        check_counts(sp, orc, 2)
        res = sp.screen(torch.from_numpy(y).cuda(), 25)
        ids, sc, eb = res.fetch(0)
        oi, os_, oc = orc.screen(y, 25)
        check_list(ids, sc, eb, oi[0], os_[0], orc, y[None, :], 0)
        assert res.stats()["reasons"] == oc


def test_decode_matches_oracle(env):
    torch, oracle, dse, W = env
    w = W.medium(1)
    sp, orc = spaces(env, w)
    rng = np.random.default_rng(3)
    for gid in list(rng.integers(0, sp.n_total, size=300)) + [0, sp.n_stored - 1, sp.n_stored, sp.n_total - 1]:
        gid = int(gid)
        assert sp.decode(gid) == orc.decode(gid)
        assert sp.expr(gid) == orc.expr(gid)


def test_determinism(env):
    torch, oracle, dse, W = env
    w = W.medium(2)
    sp, _ = spaces(env, w)
    Yd = torch.from_numpy(w["Y"]).cuda()
    a = sp.screen(Yd, w["k"]).fetch(0)
    b = sp.screen(Yd, w["k"]).fetch(0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_residual_loop_medium(env):
    """D = 1..3 with FP64 refits of the retained candidates against the
    oracle's Householder-QR loop."""
    torch, oracle, dse, W = env
    w = W.medium(0)
    sp, orc = spaces(env, w)
    y = w["Y"][0]
    ref = orc.residual_loop(y, 3, w["k"])
    r = y.copy()
    fixed = []
    for D in range(1, 4):
        res = sp.screen(torch.from_numpy(r).cuda(), w["k"])
        ids, sc, eb = res.fetch(0)
        bid, rmse, coefs, resid = sp.ls_refit(y, np.array(fixed, np.uint64), ids)
        # the oracle's pick may be an exact algebraic twin: compare RMSE
        assert abs(rmse - ref["rmse"][D - 1]) <= 1e-9 * max(ref["rmse"][D - 1], 1e-12) + 1e-13
        fixed.append(bid)
        r = resid
    assert ref["rmse"][2] < ref["rmse"][0]


@pytest.mark.parametrize("wname,D,prec", [("medium", 3, "fp32"), ("tiny", 2, "fp32"), ("medium", 2, "fp64")])
def test_residual_loop_on_device(env, wname, D, prec):
    """dse_residual_loop (screen, refit and residual chained on the device)
    against the oracle's loop (RMSE per iteration; the pick may be an exact
    algebraic twin) and against the host-driven sequence of the same calls
    (identical picks, RMSEs and SIS subspaces)."""
    torch, oracle, dse, W = env
    w = getattr(W, wname)(0)
    sp, orc = spaces(env, w)
    y = w["Y"][0]
    k = w["k"]
    p = dse.PREC_FP64 if prec == "fp64" else dse.PREC_FP32
    ref = orc.residual_loop(y, D, k)
    ids = np.zeros((D, k), np.uint64)
    resid = np.zeros(len(y))
    out = sp.residual_loop(y, D, k, precision=p, sis_ids=ids, residual=resid)
    for d in range(D):
        assert abs(out["rmse"][d] - ref["rmse"][d]) <= 1e-9 * max(ref["rmse"][d], 1e-12) + 1e-13, d
        assert out["stats"][d]["screened"] == sp.n_total
        assert sum(out["stats"][d]["reasons"].values()) == sp.n_total
    # the first subspace is the oracle's screen of y (same top-k set up to ties)
    n1 = int(np.sum(ids[0] != np.iinfo(np.uint64).max))
    assert n1 == k
    oids, osc, _ = orc.screen(y, k)
    sc1, why = orc.score_ids(y[None, :], ids[0][:n1])
    assert np.all(why == 0)
    sk = osc[0][-1]
    assert np.all(sc1[:, 0] >= sk * (1 - 1e-5))
    above = {int(i) for i, s_ in zip(oids[0], osc[0]) if s_ > sk * (1 + 1e-5)}
    assert above <= {int(i) for i in ids[0][:n1]}
    # the host-driven sequence of the same calls gives the same loop
    r = y.copy()
    fixed = []
    for d in range(D):
        res = sp.screen(r, k, precision=p)
        hids, hsc, heb = res.fetch(0)
        # the loop takes every retained score from the pair sums it needs for
        # the refit, a single screen from the FP32 re-score where that is
        # within the tolerance: the same set, in an order that may differ
        # inside the scores' bounds
        np.testing.assert_array_equal(np.sort(hids), np.sort(ids[d][:len(hids)]))
        bid, rmse, coefs, resid_h = sp.ls_refit(y, np.array(fixed, np.uint64), hids)
        assert bid == out["chosen"][d]
        assert rmse == out["rmse"][d]
        np.testing.assert_array_equal(coefs, np.array(out["coefs"][d]))
        fixed.append(bid)
        r = resid_h
    np.testing.assert_array_equal(resid, r)


def test_timing_flags(env):
    """DSE_FLAG_TIMING_MAIN times the product/quotient group alone (two
    events per screen); DSE_FLAG_TIMING every group; neither changes the
    result."""
    torch, oracle, dse, W = env
    w = W.medium(0)
    sp, _ = spaces(env, w)
    Yd = torch.from_numpy(w["Y"]).cuda()
    base = sp.screen(Yd, w["k"])
    ids0, sc0, _ = base.fetch(0)
    main = sp.screen(Yd, w["k"], flags=dse.FLAG_TIMING_MAIN)
    ids1, sc1, _ = main.fetch(0)
    km = main.stats()["kernel_ms"]
    assert km[1] > 0 and km[0] == 0 and km[2] == 0 and km[3] == 0
    full = sp.screen(Yd, w["k"], flags=dse.FLAG_TIMING)
    ids2, sc2, _ = full.fetch(0)
    assert all(x > 0 for x in full.stats()["kernel_ms"])
    for ids, sc in ((ids1, sc1), (ids2, sc2)):
        np.testing.assert_array_equal(ids, ids0)
        np.testing.assert_array_equal(sc, sc0)
    out = sp.residual_loop(w["Y"][0], 2, w["k"], flags=dse.FLAG_TIMING_MAIN)
    for st in out["stats"]:
        assert st["kernel_ms"][1] > 0 and st["kernel_ms"][0] == 0
