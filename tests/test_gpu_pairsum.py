"""The re-score's and the refits' column sums in FP32-pair arithmetic (with
the FP64 fallback), through the C ABI, against the CPU FP64 oracle, on
features that stress the pair format: magnitudes from 1e-12 to 1e12, mixed
signs, every operator, and a primary that is constant to 1e-10 relative
(its sums fall back to FP64).

Bars: every returned score within 1e-5 relative of the oracle's and within
its reported bound; top-k sets equal apart from ties; loop RMSEs within 1e-9
relative of the oracle's loop (the pick may be an exact algebraic twin).
"""
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

    return torch, oracle, dse


def stress_data(seed, N=300):
    rng = np.random.default_rng(seed)
    cols = [
        rng.uniform(0.5, 2.0, N) * 1e12,
        rng.uniform(0.5, 2.0, N) * 1e-12,
        rng.uniform(-1.0, 1.0, N),
        rng.uniform(1.0, 3.0, N),
        1000.0 + 1e-7 * rng.uniform(0.0, 1.0, N),  # constant to 1e-10 relative
        -rng.uniform(0.1, 5.0, N) * 1e6,
        rng.uniform(0.2, 1.2, N),
        rng.standard_normal(N) * 1e-3 + 0.5,
    ]
    X = np.stack(cols)
    y = (cols[3] * cols[6] / cols[7] + 1e-12 * cols[0] * cols[2] + 0.03 * rng.standard_normal(N))
    return X, y


ALL_OPS = (1 << 12) - 1


@pytest.mark.parametrize("seed", [0, 1])
def test_pair_sums_screen_extreme_scales(env, seed):
    torch, oracle, dse = env
    X, y = stress_data(seed)
    sp = dse.Space(torch.from_numpy(X).cuda(), None, ALL_OPS, 2)
    orc = oracle.Space(X, None, ALL_OPS, 2)
    assert sp.n_total == orc.total_candidates
    for k in (50, 2000):
        res = sp.screen(torch.from_numpy(y).cuda(), k)
        ids, sc, eb = res.fetch(0)
        oids, osc, ocnt = orc.screen(y, k)
        ge._check_topk(ids, sc, eb, oids[0], osc[0], orc, y[None, :], 0, tol=1e-5)
        assert res.stats()["reasons"] == ocnt


@pytest.mark.parametrize("seed", [0, 3])
def test_pair_sums_residual_loop_extreme_scales(env, seed):
    torch, oracle, dse = env
    X, y = stress_data(seed)
    sp = dse.Space(torch.from_numpy(X).cuda(), None, ALL_OPS, 2)
    orc = oracle.Space(X, None, ALL_OPS, 2)
    D, k = 3, 400
    ref = orc.residual_loop(y, D, k)
    out = sp.residual_loop(y, D, k)
    for d in range(D):
        assert abs(out["rmse"][d] - ref["rmse"][d]) <= 1e-9 * max(ref["rmse"][d], 1e-12) + 1e-13, d
    # the refit entry point on the same subspace gives the same pick
    ids = np.zeros((D, k), np.uint64)
    out2 = sp.residual_loop(y, D, k, sis_ids=ids)
    assert list(out2["chosen"]) == list(out["chosen"])
    bid, rmse, coefs, resid = sp.ls_refit(y, np.array([], np.uint64), ids[0])
    assert bid == out["chosen"][0] and rmse == out["rmse"][0]
