"""Failure detection without a GPU fault.

* A bounded device wait on a barrier that nothing completes runs out and the
  library reports DSE_ETIMEOUT; the context stays usable (a screen right
  after it matches the oracle).  The same bounded poll loop guards every
  pipelined kernel's waits.
* A simulated allocation failure (host-side hook) at every allocation of a
  space build and of a screen returns DSE_ENOMEM cleanly, and the library
  works normally once the hook is off.
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
    from paper_2602_06986_gb300 import workloads as W

    return torch, oracle, dse, W


def _tiny_screen_matches_oracle(env):
    torch, oracle, dse, W = env
    w = W.tiny(1)
    kw = dict(unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    sp = dse.Space(torch.from_numpy(w["X"]).cuda(), w["units"], w["op_mask"], w["max_rung"], **kw)
    orc = oracle.Space(w["X"], w["units"], w["op_mask"], w["max_rung"], **kw)
    res = sp.screen(torch.from_numpy(w["Y"]).cuda(), w["k"])
    ids, sc, eb = res.fetch(0)
    oids, osc, ocnt = orc.screen(w["Y"], w["k"])
    ge._check_topk(ids, sc, eb, oids[0], osc[0], orc, w["Y"], 0)
    assert res.stats()["reasons"] == ocnt
    res.free()
    sp.free()


def test_bounded_wait_runs_out(env):
    torch, oracle, dse, W = env
    assert dse.check_wait(2000, arrive=False) == dse.ETIMEOUT
    assert "timed out" in dse.lib().dse_last_error().decode()
    assert dse.check_wait(2000, arrive=True) == dse.OK
    # the context is still usable
    _tiny_screen_matches_oracle(env)
    assert dse.check_wait(10, arrive=False) == dse.ETIMEOUT
    _tiny_screen_matches_oracle(env)


def test_simulated_allocation_failures(env):
    torch, oracle, dse, W = env
    w = W.tiny(0)
    kw = dict(unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    Xd = torch.from_numpy(w["X"]).cuda()
    Yd = torch.from_numpy(w["Y"]).cuda()
    try:
        # every allocation of a space build in turn
        build_failures = 0
        for after in range(1000):
            dse.debug_fail_alloc(after)
            try:
                sp = dse.Space(Xd, w["units"], w["op_mask"], w["max_rung"], **kw)
            except dse.DseError as e:
                assert e.status == dse.ENOMEM, e
                assert "simulated" in str(e)
                build_failures += 1
                continue
            sp.free()
            break
        else:
            pytest.fail("the build never completed")
        assert build_failures >= 1
        # every allocation of a screen in turn, on a good space
        dse.debug_fail_alloc(-1)
        sp = dse.Space(Xd, w["units"], w["op_mask"], w["max_rung"], **kw)
        screen_failures = 0
        for after in range(1000):
            dse.debug_fail_alloc(after)
            try:
                res = sp.screen(Yd, w["k"])
                res.fetch(0)
                res.free()
            except dse.DseError as e:
                assert e.status == dse.ENOMEM, e
                screen_failures += 1
                continue
            break
        else:
            pytest.fail("the screen never completed")
        assert screen_failures >= 1
        sp.free()
    finally:
        dse.debug_fail_alloc(-1)
    _tiny_screen_matches_oracle(env)
