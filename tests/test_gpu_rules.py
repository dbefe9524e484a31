"""GPU parity of the user rules on variable combinations / functional forms
and of score-window redundancy removal, through the C ABI, against the CPU
FP64 oracle.

Bars: stored features, candidate counts and reason counts bit-exact; returned
lists as in the plain screen (scores within 1e-5 relative and within the
reported bound, sets equal apart from ties within 1e-5 * s_k); redundancy
decisions equal (the oracle reports how close its correlations came to the
threshold).
"""
import numpy as np
import pytest

import __graft_entry__ as ge

pytestmark = pytest.mark.gpu

TOL = 1e-5
TAU = 1e-10
SQUARE, CUBE, INV, SQRT, EXP, LOG, ADD, SUB, MUL, DIV, RDIV, ABSDIFF = range(12)


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


def rule_rows(n0, pairs, op_sets):
    pd = np.zeros(n0, np.uint64)
    for pq in pairs:
        p, q = (pq[0], pq[0]) if len(pq) == 1 else pq
        pd[p] |= np.uint64(1 << q)
    od = np.zeros(12, np.uint64)
    for o, ps in op_sets.items():
        for p in ps:
            od[o] |= np.uint64(1 << p)
    return pd, od


RULES = {
    "tiny": ([(0, 1), (2,), (3, 5)], {EXP: {4}, DIV: {6}, SQRT: {0}}),
    "medium": ([(0, 1), (2,), (3, 5), (7, 11), (12, 19)], {EXP: {4, 9}, MUL: {6}, LOG: {2}, ABSDIFF: {1, 3}}),
}


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
    slots, rs = sp.counts(max_rung)
    oslots, ors = orc.rung_counts(max_rung)
    assert slots == oslots
    for key in ("unit", "complexity", "domain", "magnitude"):
        assert rs[key] == ors[key], key


@pytest.mark.parametrize("wname,seed,prec", [("tiny", 0, "fp32"), ("tiny", 1, "fp64"), ("medium", 0, "fp32"),
                                             ("medium", 2, "fp64")])
def test_rules_parity(env, wname, seed, prec):
    torch, oracle, dse, W = env
    w = getattr(W, wname)(seed)
    pd, od = rule_rows(len(w["X"]), *RULES[wname])
    sp, orc = spaces(env, w, pair_deny=pd, op_deny=od)
    check_counts(sp, orc, w["max_rung"])
    p = dse.PREC_FP64 if prec == "fp64" else dse.PREC_FP32
    res = sp.screen(torch.from_numpy(w["Y"]).cuda(), w["k"], precision=p)
    ids, sc, eb = res.fetch(0)
    oids, osc, ocnt = orc.screen(w["Y"], w["k"])
    ge._check_topk(ids, sc, eb, oids[0], osc[0], orc, w["Y"], 0, tol=TOL)
    assert res.stats()["reasons"] == ocnt
    # the rules remove something at every rung
    assert all(orc.rung_counts(r)[1]["complexity"] > 0 for r in range(1, w["max_rung"] + 1))
    # and the unruled space is larger
    sp0, orc0 = spaces(env, w)
    assert sp0.n_stored > sp.n_stored


def test_rules_tensor_core(env):
    """The BF16x3 tcgen05 path applies the same rule test."""
    torch, oracle, dse, W = env
    w = W.tiny(7)
    X = w["X"]
    rng = np.random.default_rng(17)
    Y = np.stack([X[rng.integers(8)] * X[rng.integers(8)] / X[rng.integers(8)] + 0.05 * rng.standard_normal(100)
                  for _ in range(17)])
    pd, od = rule_rows(len(X), *RULES["tiny"])
    sp, orc = spaces(env, w, pair_deny=pd, op_deny=od)
    res = sp.screen(torch.from_numpy(Y).cuda(), 40, precision=dse.PREC_BF16X3)
    st = res.stats()
    assert st["precision_used"] == dse.PREC_BF16X3
    oids, osc, ocnt = orc.screen(Y, 40)
    assert st["reasons"] == ocnt
    for l in range(len(Y)):
        ids, sc, eb = res.fetch(l)
        ge._check_topk(ids, sc, eb, oids[l], osc[l], orc, Y, l, tol=TOL)


def test_rules_limits(env):
    torch, oracle, dse, W = env
    rng = np.random.default_rng(0)
    X = rng.uniform(0.5, 2.0, size=(65, 16))
    with pytest.raises(dse.DseError):
        dse.Space(X, None, (1 << MUL), 1, pair_deny=np.zeros(65, np.uint64))
    # the same space without rules builds
    dse.Space(X, None, (1 << MUL), 1).free()


@pytest.mark.parametrize("wname,seed,prec,k", [("tiny", 0, "fp32", 100), ("tiny", 2, "fp64", 40),
                                               ("medium", 0, "fp32", 1000), ("medium", 1, "fp32", 150)])
def test_dedup_parity(env, wname, seed, prec, k):
    torch, oracle, dse, W = env
    w = getattr(W, wname)(seed)
    sp, orc = spaces(env, w)
    p = dse.PREC_FP64 if prec == "fp64" else dse.PREC_FP32
    res = sp.screen(torch.from_numpy(w["Y"]).cuda(), k, precision=p, dedup_tau=TAU)
    ids, sc, eb = res.fetch(0)
    oids, osc, ored, margin = orc.screen_dedup(w["Y"], k, TAU)
    assert margin > 1e-12
    ge._check_topk(ids, sc, eb, oids[0], osc[0], orc, w["Y"], 0, tol=TOL)
    st = res.stats()
    assert st["redundant"] > 0 and st["dedup_rounds"] >= 1
    # no two returned candidates are equivalent
    V = np.array([orc.candidate(int(i))[0] for i in ids])
    Z = V - V.mean(axis=1, keepdims=True)
    Z /= np.linalg.norm(Z, axis=1, keepdims=True)
    R = np.abs(Z @ Z.T) - np.eye(len(ids))
    assert R.max() < 1 - TAU


def test_dedup_multi_target_and_range(env):
    torch, oracle, dse, W = env
    w = W.tiny(4)
    X = w["X"]
    rng = np.random.default_rng(2)
    Y = np.stack([X[rng.integers(8)] * X[rng.integers(8)] / X[rng.integers(8)] + 0.05 * rng.standard_normal(100)
                  for _ in range(3)])
    sp, orc = spaces(env, w)
    a, b = 37, sp.n_total - 1234
    res = sp.screen(torch.from_numpy(Y).cuda(), 50, id_begin=a, id_end=b, dedup_tau=TAU)
    oids, osc, ored, margin = orc.screen_dedup(Y, 50, TAU, id_begin=a, id_end=b)
    assert margin > 1e-12
    for l in range(3):
        ids, sc, eb = res.fetch(l)
        assert np.all((ids >= a) & (ids < b))
        ge._check_topk(ids, sc, eb, oids[l], osc[l], orc, Y, l, tol=TOL)


def test_dedup_affine_copies_need_longer_lists(env):
    """Four affine copies of one variable make every sum and difference of
    them equivalent to it (16 of the 35 candidates, all at one score): when
    the k-th kept entry's score window reaches past the first list of 4k
    entries, the list has to grow (several rounds) before it is decided."""
    torch, oracle, dse, W = env
    rng = np.random.default_rng(8)
    N = 64
    x, z = rng.uniform(0.5, 2.0, N), rng.uniform(0.5, 2.0, N)
    X = np.stack([x, 2 * x + 1, 3 * x - 2, 0.5 * x + 4, z])
    y = x + 0.02 * z + 0.01 * rng.standard_normal(N)
    ops = (1 << ADD) | (1 << SUB) | (1 << MUL)
    sp = dse.Space(torch.from_numpy(X).cuda(), None, ops, 1)
    orc = oracle.Space(X, None, ops, 1)
    total = orc.total_candidates
    _, plain, _ = orc.screen(y, total)
    plain = plain[0]
    seen_multi = False
    for k in (1, 3, 8):
        res = sp.screen(torch.from_numpy(y).cuda(), k, dedup_tau=TAU)
        ids, sc, eb = res.fetch(0)
        oids, osc, ored, margin = orc.screen_dedup(y, k, TAU)
        assert margin > 1e-12
        ge._check_topk(ids, sc, eb, oids[0], osc[0], orc, y, 0, tol=TOL)
        assert [int(i) for i in ids] == [int(i) for i in oids[0]]
        rounds = res.stats()["dedup_rounds"]
        # the first list (4k entries) cannot settle the k-th kept entry when
        # its window reaches the list's end
        if 4 * k < total and osc[0][-1] - np.sqrt(2 * TAU) <= plain[4 * k - 1]:
            assert rounds >= 2, k
            seen_multi = True
        else:
            assert rounds >= 1
    assert seen_multi


def test_dedup_tau_validation(env):
    torch, oracle, dse, W = env
    w = W.tiny(0)
    sp, _ = spaces(env, w)
    for bad in (0.5, 1.0, -1e-3, float("nan")):
        with pytest.raises(dse.DseError):
            sp.screen(torch.from_numpy(w["Y"]).cuda(), 10, dedup_tau=bad)
