"""Planner settings (dse_set_tuning) change how the work is cut and ordered,
not the results: screens under non-default settings return the same lists
(apart from ties within the tolerance) and the same reason counts as under
the defaults, on the single-target, CUDA-core multi-target, tensor-core and
batched paths; and a short autotuning run on the device installs a setting
that does the same."""
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

    yield torch, oracle, dse, W
    dse.set_tuning(None)


def _space(env, w):
    torch, oracle, dse, W = env
    kw = dict(unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    return dse.Space(torch.from_numpy(w["X"]).cuda(), w["units"], w["op_mask"], w["max_rung"], **kw)


def _lists(env, sp, Y, k, **kw):
    torch = env[0]
    res = sp.screen(torch.from_numpy(np.ascontiguousarray(Y)).cuda(), k, **kw)
    out = [res.fetch(l) for l in range(res.n_lists)]
    st = res.stats()
    res.free()
    return out, st


def _same(a, b):
    (la, sa), (lb, sb) = a, b
    assert sa["reasons"] == sb["reasons"]
    for (ia, sca, _), (ib, scb, _) in zip(la, lb):
        assert len(ia) == len(ib)
        sk = min(sca[-1], scb[-1])
        strict_a = {int(i) for i, s in zip(ia, sca) if s > sk * (1 + 2 * TOL)}
        strict_b = {int(i) for i, s in zip(ib, scb) if s > sk * (1 + 2 * TOL)}
        assert strict_a <= set(int(i) for i in ib) and strict_b <= set(int(i) for i in ia)
        common = np.intersect1d(ia, ib)
        pa = {int(i): s for i, s in zip(ia, sca)}
        pb = {int(i): s for i, s in zip(ib, scb)}
        for i in common:
            assert abs(pa[int(i)] - pb[int(i)]) <= TOL * pa[int(i)] + 1e-12


@pytest.mark.parametrize("settings", [{"tile_group": 1}, {"tile_group": 16, "seed_stride": 2},
                                      {"gram_max_n": 16}])
def test_single_target_settings(env, settings):
    torch, oracle, dse, W = env
    w = W.medium(0)
    sp = _space(env, w)
    dse.set_tuning(None)
    ref = _lists(env, sp, w["Y"], 300)
    dse.set_tuning(settings)
    try:
        got = _lists(env, sp, w["Y"], 300)
    finally:
        dse.set_tuning(None)
    _same(ref, got)
    sp.free()


@pytest.mark.parametrize("settings,flags", [({"tile_group": 2, "seed_stride": 32}, 4), ({"tc_min_targets": 32}, 0),
                                            ({"gmt_group": 5}, 0), ({"gmt_cluster": 1}, 0)])
def test_multi_target_settings(env, settings, flags):
    """16 targets: the sample-by-sample tensor-core kernel (DSE_FLAG_DIRECT)
    under other tile settings; the CUDA-core path (tc_min_targets above 16),
    another tile order of the multi-target Gram kernel and that kernel with
    one CTA per tile (no clusters) against the default multi-target Gram
    screen."""
    torch, oracle, dse, W = env
    w = W.large(0, n_targets=16)
    sp = _space(env, w)
    b, e = sp.n_stored + 1_000_000, sp.n_stored + 1_600_000
    dse.set_tuning(None)
    ref = _lists(env, sp, w["Y"], 200, id_begin=b, id_end=e, precision=dse.PREC_AUTO, flags=flags)
    assert ref[1]["precision_used"] == dse.PREC_BF16X3
    assert ref[1]["binary_path"] == (dse.PATH_TENSOR if flags else dse.PATH_GRAM_MT)
    dse.set_tuning(settings)
    try:
        got = _lists(env, sp, w["Y"], 200, id_begin=b, id_end=e, precision=dse.PREC_AUTO, flags=flags)
    finally:
        dse.set_tuning(None)
    if "tc_min_targets" in settings:
        assert got[1]["precision_used"] == dse.PREC_FP32
        assert got[1]["binary_path"] == dse.PATH_CUDA_CORE
    _same(ref, got)
    sp.free()


def test_batched_job_size(env):
    torch, oracle, dse, W = env
    w = W.batched(0, n_base=4, n_folds=2, n_boot=1, n_hi=2000)
    kw = dict(unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    Xd = [torch.from_numpy(b["X"]).cuda() for b in w["bases"]]
    spaces = [dse.Space(Xd[p["base"]], w["bases"][p["base"]]["units"], w["op_mask"], w["max_rung"],
                        sample_idx=p["samples"], **kw) for p in w["problems"]]
    targets = [w["bases"][p["base"]]["y"][p["samples"]] for p in w["problems"]]
    outs = []
    for settings in (None, {"batch_job_samples": 4096}):
        dse.set_tuning(settings)
        try:
            bt = dse.Batch(spaces, targets, w["k"])
            outs.append([(bt.fetch(i), bt.stats(i)) for i in range(len(spaces))])
            bt.free()
        finally:
            dse.set_tuning(None)
    for a, b in zip(*outs):
        _same(([a[0]], a[1]), ([b[0]], b[1]))
    for sp in spaces:
        sp.free()


def test_autotune_on_device(env):
    """A short tuning run of the tensor-core class on a small 16-target
    workload installs its choice; the screen under it equals the default."""
    torch, oracle, dse, W = env
    from paper_2602_06986_gb300 import autotune as at

    w = dict(W.precision(0, n_targets=16), max_rung=2)
    sp = _space(env, w)
    Yd = torch.from_numpy(w["Y"]).cuda()

    def run():
        sp.screen(Yd, 100, precision=dse.PREC_AUTO).free()

    cache = {}
    entry = at.tune("screen_tc", sp.n_samples, 16, run, cache=cache, reps=1)
    assert len(entry["tried"]) >= 6 and all(t["seconds"] > 0 for t in entry["tried"])
    assert dse.get_tuning()["tile_group"] == 0  # defaults restored
    dse.set_tuning(None)
    ref = _lists(env, sp, w["Y"], 100, precision=dse.PREC_AUTO)
    at.apply(cache, "screen_tc", sp.n_samples, 16)
    try:
        got = _lists(env, sp, w["Y"], 100, precision=dse.PREC_AUTO)
    finally:
        dse.set_tuning(None)
    _same(ref, got)
    sp.free()
