"""Pins of the CPU FP64 oracle against things other than itself.

Each test checks the oracle against a hand derivation, a closed form, an
independent pure-Python construction, a library routine (numpy) or an
invariance of the mathematics, chosen so that a plausible slip in the oracle
(a dropped term, a swapped operand, an off-by-one in the pair decoding, a wrong
unit rule) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle.bruteforce import enumerate_bruteforce
from oracle.counts import closed_form_sizes, unit_class_counts

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQUARE, CUBE, INV, SQRT, EXP, LOG, ADD, SUB, MUL, DIV, RDIV, ABSDIFF = range(12)


def mask(*c):
    m = 0
    for x in c:
        m |= 1 << x
    return m


def unpruned_space(orc, X, ops, rung, units=None, **kw):
    kw.setdefault("fmax_max", 1e300)
    kw.setdefault("fmin_std_rel", -1.0)
    return orc.Space(X, units, mask(*ops), rung, **kw)


# ------------------------------------------------------------------ counts

@pytest.mark.parametrize("ops,rung,n0,N", [
    ((ADD, MUL, DIV, RDIV, SQUARE, CUBE, EXP), 2, 4, 16),
    ((ADD, SUB, MUL, SQUARE, CUBE), 2, 5, 12),
    ((ADD, MUL, DIV, RDIV, SQUARE), 3, 3, 8),
    ((MUL,), 2, 6, 8),
    ((SQRT, EXP), 2, 5, 8),
])
def test_counts_match_closed_form(orc, ops, rung, n0, N):
    """No pruning possible (positive data, no domain-restricted op can fail,
    huge magnitude limit, degeneracy off): every slot is valid, so |Phi_r|
    must equal the closed form."""
    rng = np.random.default_rng(7)
    X = rng.uniform(0.5, 2.0, size=(n0, N))
    S = unpruned_space(orc, X, ops, rung)
    nu = sum(1 for o in ops if o <= LOG)
    nb = len(ops) - nu
    sizes = closed_form_sizes(n0, nu, nb, rung)
    total = 0
    for r in range(rung + 1):
        slots, rs = S.rung_counts(r)
        assert rs["valid"] == slots
        total += slots
        assert total == sizes[r]
    assert S.total_candidates == sizes[rung]
    assert S.n_features == sizes[rung - 1]


def test_closed_form_golden_matches_formula():
    g = json.load(open(os.path.join(GOLDEN, "closed_form_counts.json")))
    sizes = g["sizes"]
    assert sizes["tiny: n0=8, 4 unary (sq sqrt exp log), 5 binary slots (+ - * a/b b/a), rung 2"] == [8, 180, 81278]
    for v in sizes.values():
        # |new_r| must be exactly reproducible from the previous two sizes
        for r in range(2, len(v)):
            assert v[r] > v[r - 1]


@pytest.mark.parametrize("explog_dimless", [1, 0])
@pytest.mark.parametrize("seed", [0, 1])
def test_counts_match_unit_classes(orc, explog_dimless, seed):
    """Pruning by units only: the oracle's valid counts per rung equal the
    class-wise count with Fraction exponents, which never visits a pair."""
    rng = np.random.default_rng(100 + seed)
    n0, N = 7, 10
    X = rng.uniform(0.5, 2.0, size=(n0, N))
    units = rng.integers(-2, 3, size=(n0, 3)).astype(np.int32)
    ops = (ADD, MUL, DIV, RDIV, ABSDIFF, SQUARE, CUBE, INV, SQRT, EXP)
    S = unpruned_space(orc, X, ops, 2, units=units, unit_check_addsub=1, explog_dimensionless=explog_dimless)
    ref = unit_class_counts(units, ops, 2, unit_check_addsub=True, explog_dimensionless=bool(explog_dimless))
    for r in (1, 2):
        slots, rs = S.rung_counts(r)
        assert (slots, rs["valid"]) == ref[r - 1]
        assert rs["valid"] + rs["unit"] == slots


# -------------------------------------------------------- enumeration order

def _hand_case(orc, case):
    g = json.load(open(os.path.join(GOLDEN, "tiny_space_2primaries.json")))
    c = g[case]
    X = np.array([[0.7, 1.3, 1.9, 0.6], [1.1, 0.8, 1.7, 1.4]])
    S = unpruned_space(orc, X, (SQUARE, ADD), 2, units=np.array(c["units"], np.int32))
    return S, c


@pytest.mark.parametrize("case", ["dimensionless", "unit_clash"])
def test_hand_enumerated_space(orc, case):
    S, c = _hand_case(orc, case)
    assert S.n_features == len(c["stored"])
    assert [S.expr(i) for i in range(S.n_features)] == c["stored"]
    n2 = S.rung_slots(2)
    assert n2 == len(c["rung2"])
    got = [S.expr(S.n_features + p) for p in range(n2)]
    assert got == c["rung2"]
    valid = [S.candidate(S.n_features + p)[1] == 0 for p in range(n2)]
    assert valid == c["rung2_unit_valid"]
    if "rung1_slots" in c:
        slots, rs = S.rung_counts(1)
        assert (slots, rs["valid"]) == (c["rung1_slots"], c["rung1_valid"])


@pytest.mark.parametrize("n0,rung,ops,dims,seed", [
    (4, 2, (ADD, SUB, MUL, DIV, RDIV, ABSDIFF, SQUARE, CUBE, INV, SQRT, EXP), 2, 0),
    (3, 2, (SUB, DIV, SQRT), 1, 1),
    (4, 2, (RDIV, ABSDIFF, EXP, LOG), 2, 2),
    (2, 3, (ADD, DIV, SQUARE), 1, 3),
])
def test_bruteforce_enumeration(orc, n0, rung, ops, dims, seed):
    """The oracle's decoding of every flat index (integer bisection on the
    pair triangle) and its unit rule against explicit expression trees with
    Fraction exponents.  Data positive and |a-b|, a-b never feed a
    domain-restricted op at the last rung here unless the op set has none."""
    rng = np.random.default_rng(seed)
    N = 6
    X = rng.uniform(0.5, 2.0, size=(n0, N))
    units = rng.integers(-1, 2, size=(n0, dims)).astype(np.int32)
    # keep the unit pruning the only pruning: degeneracy off, huge magnitude,
    # and domain tests cannot fail for positive data at rung 1; at the last
    # rung a domain failure is reported as 'domain', which we accept only for
    # slots the brute force marks unit-valid.
    S = unpruned_space(orc, X, ops, rung, units=units, unit_check_addsub=1, explog_dimensionless=1)
    stored, last = enumerate_bruteforce(units, ops, rung, True, True)
    assert [S.expr(i) for i in range(S.n_features)] == [e.text for e in stored]
    assert S.rung_slots(rung) == len(last)
    for p, e in enumerate(last):
        gid = S.n_features + p
        assert S.expr(gid) == (e.text if e is not None else S.expr(gid))
        why = S.candidate(gid)[1]
        if e is None:
            assert why == 1, (p, S.expr(gid))
        else:
            assert why in (0, 3), (p, e.text, why)
            assert S.expr(gid) == e.text


def test_unit_invalid_strings_still_decode(orc):
    """Unit-invalid slots decode to the expression the brute force would build
    without the unit check."""
    rng = np.random.default_rng(5)
    units = np.array([[1], [0], [2]], np.int32)
    X = rng.uniform(0.5, 2.0, size=(3, 5))
    ops = (ADD, SUB, MUL)
    S = unpruned_space(orc, X, ops, 2, units=units)
    stored, last_checked = enumerate_bruteforce(units, ops, 2, True, True)
    # the unchecked enumeration of the last rung from the same stored set
    from oracle.bruteforce import _binary
    begin = [i for i, e in enumerate(stored) if e.rung == 1][0]
    texts = []
    for i in range(begin, len(stored)):
        for j in range(i):
            for op in ops:
                texts.append(_binary(op, stored[i], stored[j], False, 2).text)
    assert [S.expr(S.n_features + p) for p in range(S.rung_slots(2))] == texts


# -------------------------------------------------------------------- score

def test_pearson_hand_value(orc):
    g = json.load(open(os.path.join(GOLDEN, "pearson_hand.json")))
    X = np.array([g["v"], [0.3, 0.9, 0.1, 0.5]])
    S = unpruned_space(orc, X, (MUL,), 1)
    sc, why = S.score_ids(np.array(g["y"]), [0])
    assert why[0] == 0
    assert abs(sc[0, 0] - g["score_num"] / math.sqrt(g["score_den_sq"])) < 1e-15


def test_score_matches_numpy_corrcoef(orc):
    rng = np.random.default_rng(11)
    X = rng.uniform(0.5, 2.0, size=(6, 40))
    Y = rng.standard_normal((3, 40))
    S = orc.Space(X, None, mask(ADD, SUB, MUL, DIV, RDIV, SQRT, LOG), 2)
    ids = rng.choice(S.total_candidates, size=300, replace=False).astype(np.uint64)
    sc, why = S.score_ids(Y, ids)
    checked = 0
    for n, gid in enumerate(ids):
        v, w = S.candidate(int(gid))
        assert w == why[n]
        if w:
            continue
        for t in range(3):
            ref = abs(np.corrcoef(v, Y[t])[0, 1])
            assert abs(sc[n, t] - ref) <= 1e-12 * max(ref, 1e-3)
        checked += 1
    assert checked > 150


def test_score_affine_invariance(orc):
    """score(alpha*y + beta) == score(y), and a primary that is an affine map
    of another gets the same score as it."""
    rng = np.random.default_rng(12)
    X = rng.uniform(0.5, 2.0, size=(5, 64))
    X = np.vstack([X, -3.5 * X[2] + 7.25])
    y = rng.standard_normal(64)
    S = orc.Space(X, None, mask(ADD, MUL, DIV, RDIV, SQUARE), 2)
    ids = np.arange(0, S.total_candidates, 7, dtype=np.uint64)
    s1, w1 = S.score_ids(y, ids)
    s2, w2 = S.score_ids(-0.25 * y + 3.0, ids)
    ok = w1 == 0
    assert ok.sum() > 100
    assert np.all(w1 == w2)
    # relative to the score, floored at 1e-2: a score near 0 is an absolute
    # cancellation of size ~1e-16 in the numerator
    assert np.max(np.abs(s1[ok] - s2[ok]) / np.maximum(s1[ok], 1e-2)) < 1e-12
    s, _ = S.score_ids(y, [2, 5])
    assert abs(s[0, 0] - s[1, 0]) < 1e-12


def test_aggregated_equals_per_target_for_one_target(orc):
    rng = np.random.default_rng(13)
    X = rng.uniform(0.5, 2.0, size=(5, 30))
    y = rng.standard_normal(30)
    S = orc.Space(X, None, mask(ADD, SUB, MUL, DIV, RDIV), 2)
    a_ids, a_sc, _ = S.screen(y, 50, mode="aggregated")
    p_ids, p_sc, _ = S.screen(y, 50, mode="per_target")
    assert np.array_equal(a_ids[0], p_ids[0])
    assert np.allclose(a_sc[0], p_sc[0], rtol=1e-14, atol=0)


def test_topk_equals_full_ranking(orc):
    """The streaming per-thread top-k equals a full ranking of all valid
    candidates by numpy lexsort on (score desc, id asc)."""
    rng = np.random.default_rng(14)
    X = rng.uniform(0.5, 2.0, size=(5, 25))
    Y = rng.standard_normal((2, 25))
    S = orc.Space(X, None, mask(ADD, SUB, MUL, DIV, RDIV, SQRT), 2)
    ids = np.arange(S.total_candidates, dtype=np.uint64)
    sc, why = S.score_ids(Y, ids)
    for k in (1, 37, 5000):
        got_ids, got_sc, cnt = S.screen(Y, k)
        assert cnt["valid"] == int((why == 0).sum())
        for t in range(2):
            v = why == 0
            order = np.lexsort((ids[v], -sc[v, t]))
            ref = ids[v][order][:k]
            assert np.array_equal(got_ids[t], ref)
            assert np.array_equal(got_sc[t], sc[v, t][order][:k])


def test_planted_formula_recovered_noise_free(orc):
    from paper_2602_06986_gb300 import workloads as W

    w = W.tiny(seed=3, noise=0.0)
    S = orc.Space(w["X"], w["units"], w["op_mask"], 2, unit_check_addsub=1, explog_dimensionless=0)
    ids, sc, _ = S.screen(w["Y"], 10)
    assert 1.0 - sc[0][0] < 1e-14
    top = [S.expr(int(i)) for i, s in zip(ids[0], sc[0]) if 1.0 - s < 1e-13]
    assert w["planted"] in top
    # every member of the top tie group is an algebraic rewrite of 2*x1*x3/x5^2
    X = w["X"]
    ref = X[1] * X[3] / X[5] ** 2
    for i, s in zip(ids[0], sc[0]):
        if 1.0 - s < 1e-13:
            v, _ = S.candidate(int(i))
            c = np.polyfit(ref, v, 1)
            assert np.allclose(np.polyval(c, ref), v, rtol=1e-12, atol=1e-12)


# -------------------------------------------------------------------- masks

def test_domain_magnitude_realised_reasons(orc):
    N = 8
    x0 = np.array([-1.0, -0.6, -0.004, 0.2, 0.5, 0.9, 1.2, 1.5])  # crosses zero
    x1 = np.linspace(0.5, 2.0, N)           # positive
    x2 = np.linspace(81.0, 90.0, N)         # exp(x2) beyond the domain limit
    X = np.vstack([x0, x1, x2])
    S = orc.Space(X, None, mask(SQRT, EXP, LOG, MUL, DIV, RDIV, INV), 1, fmax_max=100.0, fmin_std_rel=1e-8)
    nf = S.n_features
    names = {S.expr(nf + p): S.candidate(nf + p)[1] for p in range(S.rung_slots(1))}
    assert names["log(x0)"] == 3 and names["sqrt(x0)"] == 3
    assert names["log(x1)"] == 0 and names["sqrt(x1)"] == 0
    assert names["exp(x2)"] == 3              # max > 80
    assert names["exp(x1)"] == 0              # e^2 < log(100) bound holds: max 2 <= log(100)
    assert names["inv(x1)"] == 0
    # 1/x0: min|x0| = 0.004 > 0, but 1/min|x0| = 250 > 100 -> magnitude
    assert min(abs(x0)) > 0 and 1.0 / min(abs(x0)) > 100.0
    assert names["inv(x0)"] == 4
    # x2*x1 bound = 90*2 = 180 > 100 -> magnitude; x1*x0 bound 3 <= 100
    assert names["(x2*x1)"] == 4 and names["(x1*x0)"] == 0
    # (x1/x0): 2/0.004 > 100 -> magnitude; (x0/x1): 1.5/0.5 <= 100
    assert names["(x1/x0)"] == 4 and names["(x0/x1)"] == 0


def test_exact_reciprocal_product_is_degenerate(orc):
    rng = np.random.default_rng(15)
    X = rng.uniform(0.5, 2.0, size=(2, 32))
    S = orc.Space(X, None, mask(MUL, DIV, RDIV), 2, fmin_std_rel=1e-8)
    nf = S.n_features
    found = False
    for p in range(S.rung_slots(2)):
        e = S.expr(nf + p)
        if e in ("((x1/x0)*(x0/x1))", "((x0/x1)*(x1/x0))"):
            assert S.candidate(nf + p)[1] == 5
            found = True
    assert found


# ------------------------------------------------------------ residual loop

def test_residual_loop_recovers_two_terms(orc):
    """Noise-free y = c1*fa + c2*fb: D=2 picks columns spanning fa and fb and
    the RMSE vanishes; the coefficients equal numpy lstsq on those columns."""
    rng = np.random.default_rng(16)
    N, n0 = 200, 6
    X = rng.lognormal(0.0, 0.5, size=(n0, N))
    fa = X[0] * X[1] / X[2] ** 2
    fb = (X[3] / X[4]) * np.sqrt(X[5])
    y = 1.5 * fa - 0.8 * fb + 0.3
    S = orc.Space(X, None, mask(*range(12)), 2)
    out = S.residual_loop(y, 3, 200)
    assert out["rmse"][1] < 1e-10 * y.std()
    assert out["rmse"][0] > 1e-3
    cols = [S.candidate(int(i))[0] for i in out["ids"][:2]]
    A = np.column_stack([np.ones(N)] + cols)
    beta = np.linalg.lstsq(A, y, rcond=None)[0]
    assert np.allclose(beta, out["coefs"][1][:3], rtol=1e-8, atol=1e-10)
    # the chosen two columns reproduce fa and fb up to scale
    for f in (fa, fb):
        B = np.column_stack([np.ones(N)] + cols)
        r = f - B @ np.linalg.lstsq(B, f, rcond=None)[0]
        assert np.sqrt(np.mean(r ** 2)) < 1e-9 * f.std()


def test_residual_loop_first_pick_is_top_sis(orc):
    rng = np.random.default_rng(17)
    X = rng.uniform(0.5, 2.0, size=(5, 80))
    y = X[0] * X[1] + 0.05 * rng.standard_normal(80)
    S = orc.Space(X, None, mask(ADD, SUB, MUL, DIV, RDIV), 2)
    out = S.residual_loop(y, 2, 50)
    ids, sc, _ = S.screen(y, 50)
    assert np.array_equal(out["sis"][0], ids[0])
    # the smallest one-feature RMSE belongs to the largest |r|; algebraic
    # rewrites of the same feature tie to ~1e-16, so any of them may win
    pick = list(ids[0]).index(out["ids"][0])
    assert sc[0][0] - sc[0][pick] < 1e-13
    # one-feature LS RMSE from the correlation: sqrt(Syy (1 - r^2) / N)
    r = sc[0][pick]
    yc = y - y.mean()
    assert abs(out["rmse"][0] - math.sqrt(np.sum(yc ** 2) * (1 - r * r) / 80)) < 1e-12


def test_threshold_margin_report_pin():
    """The margin report measures the distance to the threshold: a square
    whose a-priori bound sits 1e-6 (relative) under fmax_max."""
    import oracle

    X = np.array([[1.0, -2.0, 1.5, 0.5], [1.0, 2.0, 3.0, 4.0]])
    fmax = 4.0 * (1 + 1e-6)
    S = oracle.Space(X, None, oracle.op_mask(oracle.SQUARE), 1, fmax_max=fmax)
    m = S.margins(1)
    assert m["slots"] == 2
    # square of row 1 has bound 16 > fmax (decided, margin 3); row 0's bound 4
    assert abs(m["magnitude"] - (fmax - 4.0) / fmax) < 1e-15


@pytest.mark.parametrize("name,seed,samples", [("tiny", 0, None), ("tiny", 1, None), ("tiny", 2, None),
                                               ("medium", 0, 300000), ("precision", 0, 200000),
                                               ("large", 0, 200000)])
def test_threshold_margins_of_committed_seeds(name, seed, samples):
    """Every magnitude, exp-domain and realised decision of the committed
    seeds (all build rungs, and the screened rung in full or on its first
    slots) is at least 1e-9 (relative) away from its threshold, so FP64
    library differences of an ulp cannot flip a mask between the oracle and
    the CUDA path."""
    import oracle
    from paper_2602_06986_gb300 import workloads as W

    w = getattr(W, name)(seed)
    S = oracle.Space(w["X"], w["units"], w["op_mask"], w["max_rung"], unit_check_addsub=w["unit_check_addsub"],
                     explog_dimensionless=w["explog_dimensionless"])
    for r in range(1, w["max_rung"] + 1):
        end = None if (samples is None or r < w["max_rung"]) else samples
        m = S.margins(r, 0, end) if end is not None else S.margins(r)
        assert m["slots"] > 0
        for key in ("magnitude", "exp_domain", "realised"):
            assert m[key] > 1e-9, (name, seed, r, key, m[key])


def _l0_space():
    import oracle
    from paper_2602_06986_gb300 import workloads as W

    w = W.tiny(0)
    S = oracle.Space(w["X"], w["units"], w["op_mask"], w["max_rung"], unit_check_addsub=w["unit_check_addsub"],
                     explog_dimensionless=w["explog_dimensionless"])
    return S, w


@pytest.mark.parametrize("D", [1, 2, 3])
def test_l0_search_brute_force_lstsq(D):
    """The exhaustive L0 search against numpy.linalg.lstsq over every
    D-subset of a small subspace (independent arithmetic)."""
    import itertools

    S, w = _l0_space()
    rng = np.random.default_rng(D)
    y = w["Y"][0] + 0.3 * rng.standard_normal(w["X"].shape[1])
    ids = np.sort(rng.choice(S.total_candidates, size=40, replace=False)).astype(np.uint64)
    vals = []
    for g in ids:
        v, why = S.candidate(int(g))
        vals.append(v if why == 0 else None)
    keep = [i for i, v in enumerate(vals) if v is not None][:11]
    ids = ids[keep]
    cols = np.stack([vals[i] for i in keep])
    ref = []
    for tup in itertools.combinations(range(len(ids)), D):
        A = np.column_stack([np.ones(cols.shape[1])] + [cols[t] for t in tup])
        beta, *_ = np.linalg.lstsq(A, y, rcond=None)
        if np.linalg.matrix_rank(A) < A.shape[1]:
            continue
        ref.append((float(np.sqrt(np.mean((y - A @ beta) ** 2))), tup))
    ref.sort()
    pos, rm = S.l0_search(y, ids, D, 10)
    assert len(pos) == 10
    for i in range(10):
        assert abs(rm[i] - ref[i][0]) <= 1e-12 * ref[i][0] + 1e-15
    # same subsets apart from RMSE ties
    got = {tuple(p) for p, r in zip(pos.tolist(), rm) if r < ref[9][0] * (1 - 1e-9)}
    want = {t for r, t in ref[:10] if r < ref[9][0] * (1 - 1e-9)}
    assert got == want


def test_l0_search_special_cases():
    """D = 1 is the largest |Pearson| (RMSE = std(y) sqrt(1 - r^2)); a
    noise-free two-term model is recovered with RMSE ~ 0; the best RMSE does
    not grow with D."""
    S, w = _l0_space()
    y0 = w["Y"][0]
    ids, sc, _ = S.screen(y0, 30)
    ids = np.sort(ids[0])
    cols = np.stack([S.candidate(int(g))[0] for g in ids])
    r = np.array([np.corrcoef(c, y0)[0, 1] for c in cols])
    pos, rm = S.l0_search(y0, ids, 1, 3)
    best = int(np.argmax(np.abs(r)))
    assert abs(abs(r[pos[0][0]]) - abs(r[best])) <= 1e-12
    assert abs(rm[0] - np.std(y0) * np.sqrt(1 - r[best] ** 2)) <= 1e-10 * np.std(y0)
    # planted: y = 1.5 + 2 c_a - 0.7 c_b
    a, b = 3, 17
    yp = 1.5 + 2.0 * cols[a] - 0.7 * cols[b]
    pos2, rm2 = S.l0_search(yp, ids, 2, 4)
    assert rm2[0] <= 1e-10 * np.std(yp)
    assert tuple(pos2[0]) == (a, b) or rm2[0] <= 1e-12 * np.std(yp)
    best = [S.l0_search(y0, ids, D, 1)[1][0] for D in (1, 2, 3)]
    assert best[2] <= best[1] <= best[0]


# --------------------------------------------- user rules (variable combinations)

def _rule_rows(n0, pairs, op_sets):
    """uint64 rule rows; each pair is set in one direction only (the oracle
    makes the relation symmetric)."""
    pd = np.zeros(n0, np.uint64)
    for pq in pairs:
        p, q = (pq[0], pq[0]) if len(pq) == 1 else pq
        pd[p] |= np.uint64(1 << q)
    od = np.zeros(12, np.uint64)
    for o, ps in op_sets.items():
        for p in ps:
            od[o] |= np.uint64(1 << p)
    return pd, od


@pytest.mark.parametrize("n0,rung,ops,dims,seed,pairs,op_sets", [
    (4, 2, (ADD, SUB, MUL, DIV, SQUARE, SQRT, EXP), 1, 0, [(0, 1), (2,)], {EXP: {3}, MUL: {0}}),
    (3, 3, (ADD, DIV, SQUARE), 1, 1, [(2, 0)], {SQUARE: {1}}),
    (5, 2, (MUL, RDIV, ABSDIFF, INV, LOG), 2, 2, [(1,), (3,), (4, 0)], {ABSDIFF: {2}}),
    (4, 2, (ADD, MUL, DIV, RDIV, CUBE), 0, 3, [(0,), (1,), (2,), (3,)], {}),
])
def test_rules_bruteforce(orc, n0, rung, ops, dims, seed, pairs, op_sets):
    """Rule masks against explicit expression trees: every leaf and every
    operator node of the whole tree is inspected (no incremental shortcut),
    stored features and last-rung reasons must match."""
    from oracle.bruteforce import RULE
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.5, 2.0, size=(n0, 6))
    units = rng.integers(-1, 2, size=(n0, dims)).astype(np.int32) if dims else None
    pd, od = _rule_rows(n0, pairs, op_sets)
    S = unpruned_space(orc, X, ops, rung, units=units, unit_check_addsub=1, explog_dimensionless=1,
                       pair_deny=pd, op_deny=od)
    stored, last = enumerate_bruteforce(units if dims else np.zeros((n0, 0), np.int32), ops, rung, True, True,
                                        pair_deny={frozenset(x) for x in pairs}, op_deny=op_sets)
    assert [S.expr(i) for i in range(S.n_features)] == [e.text for e in stored]
    n_rule = 0
    for p, e in enumerate(last):
        gid = S.n_features + p
        why = S.candidate(gid)[1]
        if e is None:
            assert why == 1, (p, S.expr(gid))
        elif e is RULE:
            n_rule += 1
            assert why == 2, (p, S.expr(gid), why)
        else:
            assert why in (0, 3), (p, e.text, why)
            assert S.expr(gid) == e.text
    assert n_rule > 0


def test_rules_special_cases(orc):
    """Closed forms: with every pair and every repeat forbidden no binary
    candidate survives (rung 1: all nb*T(n0) binary slots fail the rule, the
    unary ones all pass); forbidding every primary below sq removes exactly
    the sq slots; no rule at all leaves the counts unchanged."""
    rng = np.random.default_rng(7)
    n0, N = 6, 10
    X = rng.uniform(0.5, 2.0, size=(n0, N))
    ops = (ADD, SUB, MUL, DIV, RDIV, SQUARE, SQRT)
    allp = [(p, q) for p in range(n0) for q in range(p + 1)]
    pd, od = _rule_rows(n0, allp, {})
    S = unpruned_space(orc, X, ops, 1, pair_deny=pd, op_deny=od)
    slots, r = S.rung_counts(1)
    assert slots == 2 * n0 + 5 * n0 * (n0 - 1) // 2
    assert r["complexity"] == 5 * n0 * (n0 - 1) // 2 and r["valid"] == 2 * n0
    pd, od = _rule_rows(n0, [], {SQUARE: set(range(n0))})
    S2 = unpruned_space(orc, X, ops, 2, pair_deny=pd, op_deny=od)
    S0 = unpruned_space(orc, X, ops, 2)
    s2, r2 = S2.rung_counts(1)
    s0, r0 = S0.rung_counts(1)
    assert s2 == s0 and r2["complexity"] == n0 and r2["valid"] == r0["valid"] - n0
    pd, od = _rule_rows(n0, [], {})
    S3 = unpruned_space(orc, X, ops, 2, pair_deny=pd, op_deny=od)
    assert S3.rung_counts(2) == S0.rung_counts(2)


# ------------------------------------------------ redundancy removal (R16)

def _dedup_brute(orc_space, Y, tau):
    """Every valid candidate, all pairwise correlations by one numpy matrix
    product of centred unit vectors (no score window): (ids, scores,
    redundant flags, smallest | (1 - |rho|) - tau |)."""
    ids, vals = [], []
    for g in range(orc_space.total_candidates):
        v, why = orc_space.candidate(g)
        if why == 0:
            ids.append(g)
            vals.append(v)
    V = np.array(vals)
    Z = V - V.mean(axis=1, keepdims=True)
    Z /= np.linalg.norm(Z, axis=1, keepdims=True)
    y = Y - Y.mean()
    y /= np.linalg.norm(y)
    scores = np.abs(Z @ y)
    R = np.abs(Z @ Z.T)
    low = np.tril(np.ones_like(R, dtype=bool), -1)  # d < c in id order
    red = ((R >= 1.0 - tau) & low).any(axis=1)
    margin = np.abs((1.0 - R[low]) - tau).min()
    return np.array(ids, np.uint64), scores, red, margin


@pytest.mark.parametrize("k", [10, 60, 5000])
def test_dedup_brute_force(orc, k):
    """The windowed, list-doubling redundancy removal equals the plain
    definition evaluated over all pairs of valid candidates."""
    rng = np.random.default_rng(11)
    X = rng.uniform(0.5, 2.0, size=(3, 20))
    y = X[0] * X[1] / X[2] + 0.3 * X[2] + rng.normal(0, 0.05, 20)
    S = unpruned_space(orc, X, (ADD, SUB, MUL, DIV, RDIV, SQUARE, SQRT), 2)
    tau = 1e-10
    ids, scores, red, margin = _dedup_brute(S, y, tau)
    assert margin > 1e-13
    assert red.sum() > 50  # the op set makes many algebraic duplicates
    keep = np.flatnonzero(~red)
    order = sorted(keep, key=lambda i: (-scores[i], int(ids[i])))[:k]
    want = ids[order]
    got, gsc, nred, mg = S.screen_dedup(y, k, tau)
    got = got[0]
    assert len(got) == len(want) == min(k, len(keep))
    sk = scores[order[-1]]
    sure = [int(i) for i, s in zip(want, scores[order]) if s > sk + 1e-9]
    assert [int(i) for i in got[: len(sure)]] == sure
    assert set(map(int, got)) - set(map(int, want)) <= {int(i) for i, s in zip(ids, scores) if abs(s - sk) <= 1e-9}
    np.testing.assert_allclose(gsc[0], scores[order], rtol=0, atol=1e-12)
    assert mg > 1e-13


def test_dedup_affine_primary_and_identity_group(orc):
    """A primary that is an affine image of an earlier one (x1 = 3 x0 + 1) is
    redundant, and so is x1 - x0 = 2 x0 + 1; the equivalent forms of a planted
    rung-2 product collapse onto the smallest id among them."""
    rng = np.random.default_rng(3)
    x0 = rng.uniform(0.5, 2.0, 30)
    X = np.stack([x0, 3 * x0 + 1, rng.uniform(0.5, 2.0, 30), rng.uniform(0.5, 2.0, 30)])
    S = unpruned_space(orc, X, (ADD, SUB, MUL, DIV), 1)
    y = x0 + rng.normal(0, 0.01, 30)
    got = [S.expr(int(i)) for i in S.screen_dedup(y, 5)[0][0]]
    assert got[0] == "x0" and "x1" not in got and "(x1-x0)" not in got
    plain = [S.expr(int(i)) for i in S.screen(y, 5)[0][0]]
    assert {"x0", "x1", "(x1-x0)"} <= set(plain)

    Xb = rng.uniform(0.5, 2.0, size=(3, 25))
    S2 = unpruned_space(orc, Xb, (MUL, DIV, RDIV), 2)
    yb = Xb[0] * Xb[1] / Xb[2]
    ids, sc, _ = S2.screen(yb, 40)
    group = [int(i) for i, s in zip(ids[0], sc[0]) if s > 1 - 1e-12]
    assert len(group) >= 3
    d_ids, d_sc, nred, _ = S2.screen_dedup(yb, 5)
    assert int(d_ids[0][0]) == min(group) and d_sc[0][1] < 1 - 1e-6
    assert nred[0] >= len(group) - 1


def test_dedup_near_equivalent_pair_uses_full_window(orc):
    """A primary built at correlation 1 - 0.3 tau with an earlier one, against
    a target that separates their scores by about sqrt(tau): redundant by the
    definition, found only if the score window is as wide as sqrt(2 tau)."""
    rng = np.random.default_rng(5)
    N, tau = 40, 1e-10
    x0 = rng.uniform(0.5, 2.0, N)
    c0 = x0 - x0.mean()
    u0 = c0 / np.linalg.norm(c0)
    z = rng.normal(size=N)
    z -= z.mean()
    z -= (z @ u0) * u0
    z /= np.linalg.norm(z)
    eta = math.sqrt(2 * 0.3 * tau)
    x1 = x0.mean() + np.linalg.norm(c0) * (u0 + eta * z)
    X = np.stack([x0, rng.uniform(0.5, 2.0, N), x1])
    y = 2.0 * c0 / np.linalg.norm(c0) + 1.5 * z + 0.2 * rng.normal(size=N)
    S = unpruned_space(orc, X, (MUL,), 1)
    ids, scores, red, margin = _dedup_brute(S, y, tau)
    s0, s1 = scores[list(ids).index(0)], scores[list(ids).index(2)]
    assert abs(s0 - s1) > 1e-7  # outside any narrow tie window
    assert red[list(ids).index(2)] and margin > 1e-13
    got = [int(i) for i in S.screen_dedup(y, 3, tau)[0][0]]
    keep = np.flatnonzero(~red)
    want = [int(ids[i]) for i in sorted(keep, key=lambda i: (-scores[i], int(ids[i])))[:3]]
    assert got == want and 2 not in got


# ------------------------------------------------- values of every operator

def _tree_values(e, X):
    """Values of an expression tree of the brute-force enumerator, computed
    with numpy's own routines straight from the primaries (no stored rows):
    x**3 by numpy.power, 1/x by numpy.reciprocal, exp/log/sqrt by numpy."""
    if not e.kids:
        return X[e.leaf].copy()
    k = [_tree_values(c, X) for c in e.kids]
    op = e.op
    if op == SQUARE:
        return np.square(k[0])
    if op == CUBE:
        return np.power(k[0], 3)
    if op == INV:
        return np.reciprocal(k[0])
    if op == SQRT:
        return np.sqrt(k[0])
    if op == EXP:
        return np.exp(k[0])
    if op == LOG:
        return np.log(k[0])
    a, b = k  # a is the higher-id operand
    return {ADD: lambda: np.add(a, b), SUB: lambda: np.subtract(a, b), MUL: lambda: np.multiply(a, b),
            DIV: lambda: np.divide(a, b), RDIV: lambda: np.divide(b, a),
            ABSDIFF: lambda: np.abs(np.subtract(a, b))}[op]()


def _expected_reason(e, X, fmax_max, explog_arg_max):
    """Reason code of a unit-valid last-rung tree from numpy values of its
    operands (domain, then magnitude, then finiteness; the degeneracy test is
    off in these cases): the domain and magnitude readings restated per op."""
    k = [_tree_values(c, X) for c in e.kids]
    a = k[0]
    b = k[1] if len(k) > 1 else None
    Ma, ma = np.max(np.abs(a)), np.min(np.abs(a))
    op = e.op
    dom = {LOG: a.min() > 0, SQRT: a.min() >= 0, INV: ma > 0, EXP: a.max() <= 80.0,
           DIV: b is not None and np.min(np.abs(b)) > 0, RDIV: ma > 0}.get(op, True)
    if not dom:
        return 3
    if op == EXP:
        mag = a.max() <= explog_arg_max
    elif op == LOG:
        mag = True
    else:
        Mb = np.max(np.abs(b)) if b is not None else 0.0
        mb = np.min(np.abs(b)) if b is not None else 0.0
        bound = {SQUARE: Ma * Ma, CUBE: (Ma * Ma) * Ma, INV: 1.0 / ma if ma > 0 else math.inf, SQRT: math.sqrt(Ma),
                 ADD: Ma + Mb, SUB: Ma + Mb, ABSDIFF: Ma + Mb, MUL: Ma * Mb,
                 DIV: Ma / mb if mb > 0 else math.inf, RDIV: Mb / ma if ma > 0 else math.inf}[op]
        mag = bound <= fmax_max
    if not mag:
        return 4
    return 0 if np.all(np.isfinite(_tree_values(e, X))) else 5


ALL_OPS = (SQUARE, CUBE, INV, SQRT, EXP, LOG, ADD, SUB, MUL, DIV, RDIV, ABSDIFF)


@pytest.mark.parametrize("seed,n0", [(21, 3), (22, 4)])
def test_every_op_value_against_numpy_trees(orc, seed, n0):
    """Values and reason codes of every rung-2 candidate under all twelve ops
    against numpy evaluations of the brute-force enumerator's expression
    trees.  Both operand orders occur (a/b and b/a, a-b of every pair in id
    order), rung-1 features that cross zero (log x, a-b) feed the
    domain-restricted ops of rung 2, and values of both signs meet |a-b|.
    The tolerance covers one rounding per tree node plus the last-ulp
    differences between numpy's and the C library's exp/log/pow."""
    rng = np.random.default_rng(seed)
    N = 9
    X = rng.uniform(0.5, 2.0, size=(n0, N))
    S = unpruned_space(orc, X, ALL_OPS, 2)
    stored, last = enumerate_bruteforce(np.zeros((n0, 0), np.int32), ALL_OPS, 2, True, True)
    # every stored (rung <= 1) feature is valid on this data, so the stored
    # lists agree
    assert [S.expr(i) for i in range(S.n_features)] == [e.text for e in stored]
    for i, e in enumerate(stored):
        v, why = S.candidate(i)
        assert why == 0
        np.testing.assert_allclose(v, _tree_values(e, X), rtol=1e-13, atol=0)
    n_checked = {op: 0 for op in ALL_OPS}
    for p, e in enumerate(last):
        gid = S.n_features + p
        assert S.expr(gid) == e.text
        v, why = S.candidate(gid)
        ref = _tree_values(e, X)
        assert why == _expected_reason(e, X, 1e300, math.log(1e300)), (e.text, why)
        if why:
            continue
        scale = np.abs(ref) + 1e-300
        # a node's relative error can be amplified by a cancelling + - |a-b|
        # above it; bound it by the magnitudes of the tree's operands
        err = np.abs(v - ref)
        assert np.all(err <= 1e-12 * np.maximum(scale, _operand_scale(e, X))), (e.text, np.max(err / scale))
        n_checked[e.op] += 1
    assert all(c > 0 for c in n_checked.values()), n_checked


def _operand_scale(e, X):
    """Largest |value| of any node of the tree, sample by sample."""
    out = np.abs(_tree_values(e, X))
    for c in e.kids:
        out = np.maximum(out, _operand_scale(c, X))
    return out


def test_every_op_domain_and_magnitude_on_signed_data(orc):
    """Rung 1 over primaries of both signs, near zero and large: every op's
    domain and magnitude decision and every valid value against numpy.  The
    primaries are chosen so that each of log, sqrt, x^-1, exp, a/b (divisor
    b), b/a (divisor a) and the magnitude bounds of ^2, ^3, *, a/b, b/a and
    + - |a-b| fails for some operand and passes for another."""
    X = np.array([
        [-1.5, -0.3, 0.4, 1.1, 2.0, 0.7],        # x0 signed
        [0.6, 0.9, 1.3, 1.8, 2.4, 1.1],          # x1 positive
        [0.0, 0.5, 0.9, 1.4, 1.2, 0.3],          # x2 has an exact zero
        [85.0, 81.0, 90.0, 82.5, 88.0, 84.0],    # x3: exp beyond the domain limit, x3^2 > 5e3
        [1e-4, 2e-3, 0.5, 0.8, 0.3, 0.6],        # x4: tiny values, 1/x4 large
        [10.0, 12.0, 15.0, 11.0, 60.0, 14.0],    # x5: exp within the domain, above the magnitude limit
    ])
    fmax = 5e3
    S = orc.Space(X, None, mask(*ALL_OPS), 1, fmax_max=fmax, fmin_std_rel=-1.0)
    stored, last = enumerate_bruteforce(np.zeros((6, 0), np.int32), ALL_OPS, 1, True, True)
    seen = set()
    for p, e in enumerate(last):
        gid = S.n_features + p
        assert S.expr(gid) == e.text
        v, why = S.candidate(gid)
        exp_why = _expected_reason(e, X, fmax, math.log(fmax))
        assert why == exp_why, (e.text, why, exp_why)
        seen.add((e.op, why))
        if why == 0:
            ref = _tree_values(e, X)
            np.testing.assert_allclose(v, ref, rtol=4e-16, atol=0)
    for op in (LOG, SQRT, INV, EXP, DIV, RDIV):
        assert (op, 3) in seen and (op, 0) in seen, op
    for op in (SQUARE, CUBE, MUL, DIV, RDIV, INV, EXP):
        assert (op, 4) in seen, op


@pytest.mark.parametrize("n0,rung,ops,dims,seed", [
    (4, 2, ALL_OPS, 2, 0),
    (3, 2, (SUB, DIV, RDIV, SQRT, CUBE, INV), 3, 1),
    (2, 3, (ADD, DIV, SQUARE, SQRT), 1, 3),
])
def test_candidate_units_and_reasons_against_bruteforce(orc, n0, rung, ops, dims, seed):
    """Unit vectors of every candidate (stored and last rung) against the
    brute-force trees' Fraction exponents times the common denominator
    2^max_rung, and the per-candidate reason array against the value and
    reason check of each candidate one by one."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.5, 2.0, size=(n0, 7))
    units = rng.integers(-1, 2, size=(n0, dims)).astype(np.int32)
    S = unpruned_space(orc, X, ops, rung, units=units, unit_check_addsub=1, explog_dimensionless=1)
    stored, last = enumerate_bruteforce(units, ops, rung, True, True)
    den = 2 ** rung
    for i, e in enumerate(stored):
        assert list(S.candidate_unit(i)) == [int(x * den) for x in e.unit]
    why = S.reasons()
    assert len(why) == S.total_candidates
    assert np.all(why[: S.n_features] == 0)
    for p, e in enumerate(last):
        gid = S.n_features + p
        u = S.candidate_unit(gid)
        if e is None:
            assert u is None and why[gid] == 1
        else:
            assert list(u) == [int(x * den) for x in e.unit], e.text
            assert why[gid] == S.candidate(gid)[1]
    # a sub-range gives the same bytes
    a, b = S.n_features // 2, S.total_candidates - 3
    assert np.array_equal(S.reasons(a, b), why[a:b])
