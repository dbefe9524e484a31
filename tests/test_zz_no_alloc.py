"""dse_ls_refit_noalloc against dse_ls_refit, through the C ABI.

The no-alloc refit exists for callers that cannot allocate device memory
while they run: applications whose device memory belongs to their own pool
allocator or a hard budget, or that have reserved the whole device.  It must
give the same pick, RMSE, coefficients and residual as the allocating entry
point, on consecutive calls that share its fixed scratch area, for every
number of fixed descriptor columns, and refuse requests beyond its stated
limits without disturbing the calls that follow.

Collected last (file name) so that a failure here comes after every other
test has run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as ge

    ge.build()
    from paper_2602_06986_gb300 import dse
    from paper_2602_06986_gb300 import workloads as W

    w = W.medium(0)
    sp = dse.Space(torch.from_numpy(w["X"]).cuda(), w["units"], w["op_mask"], w["max_rung"],
                   unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    y = w["Y"][0]
    ids, sc, eb = sp.screen(y, w["k"]).fetch(0)
    return torch, dse, sp, y, ids


def _same(a, b):
    ida, ra, ca, resa = a
    idb, rb, cb, resb = b
    assert ida == idb
    assert abs(ra - rb) <= 1e-12 * max(abs(ra), 1e-300)
    assert np.allclose(ca, cb, rtol=1e-12, atol=0)
    assert np.allclose(resa, resb, rtol=1e-12, atol=1e-14 * np.max(np.abs(resa)))


def test_noalloc_refit_matches_refit_twice(setup):
    torch, dse, sp, y, ids = setup
    fixed = np.zeros(0, np.uint64)
    ref = sp.ls_refit(y, fixed, ids)
    _same(sp.ls_refit_noalloc(y, fixed, ids), ref)
    _same(sp.ls_refit_noalloc(y, fixed, ids), ref)
    # second descriptor slot, device-resident candidates and residual
    fixed = np.array([ref[0]], np.uint64)
    cand_d = torch.from_numpy(ids.astype(np.int64)).cuda()
    ref2 = sp.ls_refit(y, fixed, ids)
    for _ in range(2):
        res_d = torch.empty(sp.n_samples, dtype=torch.float64, device="cuda")
        got = sp.ls_refit_noalloc(y, fixed, cand_d, residual=res_d)
        _same((got[0], got[1], got[2], res_d.cpu().numpy()), ref2)


def test_noalloc_refit_rejects_oversized(setup):
    torch, dse, sp, y, ids = setup
    too_many = np.arange(16385, dtype=np.uint64)
    with pytest.raises(dse.DseError) as e:
        sp.ls_refit_noalloc(y, np.zeros(0, np.uint64), too_many)
    assert e.value.status == dse.EOVERFLOW
    assert "16384" in str(e.value)


def test_noalloc_refit_two_and_three_fixed_columns(setup):
    """The widest report and column layouts of the fixed area (n_fixed = 2
    and 3), each called twice in a row."""
    torch, dse, sp, y, ids = setup
    fixed = []
    for _ in range(4):
        f = np.array(fixed, np.uint64)
        ref = sp.ls_refit(y, f, ids)
        if len(fixed) >= 2:
            for _ in range(2):
                _same(sp.ls_refit_noalloc(y, f, ids), ref)
        fixed.append(ref[0])


def test_noalloc_refit_rejects_long_samples_then_recovers(setup):
    """A space of more samples than the area's limit is refused with
    DSE_EOVERFLOW, and the next valid call still matches dse_ls_refit."""
    torch, dse, sp, y, ids = setup
    rng = np.random.default_rng(3)
    N = 40000
    X = rng.uniform(0.5, 2.0, size=(3, N))
    big = dse.Space(torch.from_numpy(X).cuda(), None, (1 << 8) | (1 << 6), 1)
    yb = rng.standard_normal(N)
    with pytest.raises(dse.DseError) as e:
        big.ls_refit_noalloc(yb, np.zeros(0, np.uint64), np.arange(3, dtype=np.uint64))
    assert e.value.status == dse.EOVERFLOW
    assert "32768" in str(e.value)
    big.free()
    fixed = np.zeros(0, np.uint64)
    _same(sp.ls_refit_noalloc(y, fixed, ids), sp.ls_refit(y, fixed, ids))
