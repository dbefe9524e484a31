"""GPU parity of the exhaustive L0 search (dse_l0_search) against the
oracle's brute force (Householder QR of every subset): the best RMSE per
dimension within 1e-9 relative (the best subset may be an exact algebraic
twin), the returned subsets' RMSEs re-fitted by the oracle, the top lists
equal apart from ties, on SIS subspaces of the tiny and medium workloads and
on a random subspace."""
import numpy as np
import pytest

import __graft_entry__ as ge

pytestmark = pytest.mark.gpu


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


def _spaces(env, w):
    torch, oracle, dse, W = env
    kw = dict(unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    sp = dse.Space(torch.from_numpy(w["X"]).cuda(), w["units"], w["op_mask"], w["max_rung"], **kw)
    orc = oracle.Space(w["X"], w["units"], w["op_mask"], w["max_rung"], **kw)
    return sp, orc


def _oracle_rmse(orc, y, ids, pos):
    cols = np.stack([orc.candidate(int(ids[p]))[0] for p in pos])
    A = np.column_stack([np.ones(len(y))] + list(cols))
    beta, *_ = np.linalg.lstsq(A, y, rcond=None)
    return float(np.sqrt(np.mean((y - A @ beta) ** 2))), beta


@pytest.mark.parametrize("wname,n,dim", [("tiny", 60, 1), ("tiny", 60, 2), ("tiny", 60, 3), ("medium", 90, 2),
                                         ("medium", 90, 3)])
def test_l0_matches_oracle(env, wname, n, dim):
    torch, oracle, dse, W = env
    w = getattr(W, wname)(0)
    sp, orc = _spaces(env, w)
    y = w["Y"][0]
    oids, _, _ = orc.screen(y, n)
    ids = np.sort(oids[0]).astype(np.uint64)
    m = 10
    opos, orm = orc.l0_search(y, ids, dim, m)
    gpos, grm, gcf = sp.l0_search(y, ids, dim, n_top=m)
    assert len(gpos) == m
    assert abs(grm[0] - orm[0]) <= 1e-9 * orm[0] + 1e-13
    for i in range(m):
        r, beta = _oracle_rmse(orc, y, ids, gpos[i])
        assert abs(grm[i] - r) <= 1e-9 * r + 1e-13, (i, grm[i], r)
        np.testing.assert_allclose(gcf[i], beta, rtol=1e-6, atol=1e-9 * np.abs(beta).max())
        assert list(gpos[i]) == sorted(gpos[i])
    assert np.all(np.diff(grm) >= 0)
    # same top list apart from RMSE ties
    band = orm[-1] * (1 - 1e-9)
    assert {tuple(p) for p, r in zip(opos.tolist(), orm) if r < band} == \
        {tuple(p) for p, r in zip(gpos.tolist(), grm) if r < band}


def test_l0_random_subspace_and_device_ids(env):
    torch, oracle, dse, W = env
    w = W.tiny(1)
    sp, orc = _spaces(env, w)
    rng = np.random.default_rng(3)
    y = w["Y"][0] + 0.2 * rng.standard_normal(w["X"].shape[1])
    ids = np.sort(rng.choice(orc.total_candidates, size=150, replace=False)).astype(np.uint64)
    valid = np.array([orc.candidate(int(g))[1] == 0 for g in ids])
    ids = ids[valid][:70]
    opos, orm = orc.l0_search(y, ids, 2, 5)
    gpos, grm, _ = sp.l0_search(torch.from_numpy(y).cuda(), torch.from_numpy(ids.astype(np.int64)).cuda(), 2,
                                n_top=5)
    assert abs(grm[0] - orm[0]) <= 1e-9 * orm[0]
    np.testing.assert_allclose(grm, orm, rtol=1e-9)
