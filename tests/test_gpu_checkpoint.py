"""Resume of the device residual loop from chosen descriptors
(dse_loop_desc.n_fixed) and the per-iteration checkpoint built on it: an
interrupted and resumed run gives the same descriptors, RMSEs, coefficients
and SIS subspaces, to the bit, as one uninterrupted call."""
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
    from paper_2602_06986_gb300 import checkpoint as ck
    from paper_2602_06986_gb300 import dse
    from paper_2602_06986_gb300 import workloads as W

    return torch, dse, W, ck


@pytest.mark.parametrize("wname,D,prec", [("medium", 3, "fp32"), ("tiny", 3, "fp64")])
def test_resumed_loop_equals_uninterrupted(env, tmp_path, wname, D, prec):
    torch, dse, W, ck = env
    w = getattr(W, wname)(0)
    kw = dict(unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    sp = dse.Space(torch.from_numpy(w["X"]).cuda(), w["units"], w["op_mask"], w["max_rung"], **kw)
    y = w["Y"][0]
    k = min(w["k"], 500)
    p = dse.PREC_FP64 if prec == "fp64" else dse.PREC_FP32
    ids = np.zeros((D, k), np.uint64)
    full = sp.residual_loop(y, D, k, precision=p, sis_ids=ids)
    # the device loop resumed from its own first choice
    ids2 = np.full((D, k), np.iinfo(np.uint64).max, np.uint64)
    rest = sp.residual_loop(y, D, k, precision=p, sis_ids=ids2, fixed=full["chosen"][:1])
    assert rest["chosen"] == full["chosen"]
    assert rest["rmse"][1:] == full["rmse"][1:] and rest["coefs"][1:] == full["coefs"][1:]
    assert rest["rmse"][0] == full["rmse"][0]  # the recomputed fit of the fixed descriptor
    np.testing.assert_array_equal(ids2[1:], ids[1:])
    # the checkpointed run, interrupted after one iteration and resumed
    path = str(tmp_path / "loop.npz")
    part = ck.residual_loop(sp, y, D, k, path, precision=p, stop_after=1)
    assert part["chosen"] == full["chosen"][:1]
    st = ck.residual_loop(sp, y, D, k, path, precision=p)
    assert st["chosen"] == full["chosen"]
    assert st["rmse"] == full["rmse"]
    assert st["coefs"] == full["coefs"]
    for d in range(D):
        np.testing.assert_array_equal(st["sis_ids"][d], ids[d])
        assert st["stats"][d]["reasons"] == full["stats"][d]["reasons"]
    sp.free()


def test_invalid_resume_rejected(env):
    torch, dse, W, ck = env
    w = W.tiny(1)
    kw = dict(unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    sp = dse.Space(torch.from_numpy(w["X"]).cuda(), w["units"], w["op_mask"], w["max_rung"], **kw)
    y = w["Y"][0]
    # a repeated id, an id past the space, as many fixed as iterations
    for fixed, n_iter in (([3, 3], 3), ([sp.n_total], 2), ([1, 2], 2)):
        with pytest.raises(dse.DseError) as e:
            sp.residual_loop(y, n_iter, 10, fixed=fixed)
        assert e.value.status == dse.EINVAL
    sp.free()
