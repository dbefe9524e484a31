"""Per-candidate masks and unit vectors of the CUDA path against the oracle.

The screen writes the reason code it assigned to every candidate of its id
range (DSE_VALID, or the first failing test of unit, form, domain,
magnitude, realised: "Physics-Informed Constraints" and the readings of the
domain, magnitude and realised tests).  Bar: the byte arrays are equal, id by
id, to the oracle's (no -1 left: every candidate was decided by some
kernel), on every path that decides candidates: the single-target FP32 path
with the product Gram contraction and without it (sample by sample), the
plain FP64 path, the multi-target tensor-core path, and features from 1e-12
to 1e12 where the FP32 kernels escalate to FP64.  Unit vectors (exponents
over the common denominator 2^max_rung) of stored and last-rung candidates
are compared the same way.
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


def spaces(env, w, X=None):
    torch, oracle, dse, W = env
    X = w["X"] if X is None else X
    kw = dict(unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    sp = dse.Space(torch.from_numpy(X).cuda(), w["units"], w["op_mask"], w["max_rung"], **kw)
    orc = oracle.Space(X, w["units"], w["op_mask"], w["max_rung"], **kw)
    return sp, orc


def gpu_reasons(env, sp, Y, k, id_begin=0, id_end=0, **kw):
    torch = env[0]
    n = (id_end if id_end else sp.n_total) - id_begin
    why = torch.empty(n, dtype=torch.int8, device="cuda")
    res = sp.screen(torch.from_numpy(np.ascontiguousarray(Y)).cuda(), k, id_begin=id_begin, id_end=id_end,
                    reasons=why, **kw)
    st = res.stats()
    res.free()
    return why.cpu().numpy(), st


def check_equal(got, ref, st):
    assert np.all(got >= 0), f"{int(np.sum(got < 0))} candidates never decided"
    bad = np.nonzero(got != ref)[0]
    assert len(bad) == 0, f"{len(bad)} masks differ, first at offset {bad[:5]}: gpu {got[bad[:5]]} oracle {ref[bad[:5]]}"
    # the per-reason counts of the statistics are the same decisions summed
    counts = [int(np.sum(ref == c)) for c in range(6)]
    assert list(st["reasons"].values()) == counts


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_reasons_tiny_every_candidate(env, seed):
    torch, oracle, dse, W = env
    w = W.tiny(seed)
    sp, orc = spaces(env, w)
    ref = orc.reasons()
    for prec in (dse.PREC_FP32, dse.PREC_FP64):
        got, st = gpu_reasons(env, sp, w["Y"], w["k"], precision=prec)
        check_equal(got, ref, st)
    sp.free()


@pytest.mark.parametrize("flags", [0, 4])  # 4 = DSE_FLAG_DIRECT: products sample by sample
def test_reasons_medium_slice(env, flags):
    """The stored features and a 2e5-id slice of rung 2 (all slot kinds),
    with the Gram contraction of the products (flags 0) and without it."""
    torch, oracle, dse, W = env
    w = W.medium(0)
    sp, orc = spaces(env, w)
    for b, e in ((0, sp.n_stored + 3000), (sp.n_stored + 400_000, sp.n_stored + 600_000)):
        ref = orc.reasons(b, e)
        got, st = gpu_reasons(env, sp, w["Y"], 50, id_begin=b, id_end=e, flags=flags)
        check_equal(got, ref, st)
        assert np.sum(ref == 1) > 0 and np.sum(ref == 0) > 0
    sp.free()


def test_reasons_medium_fp64(env):
    torch, oracle, dse, W = env
    w = W.medium(0)
    sp, orc = spaces(env, w)
    b, e = sp.n_stored + 900_000, sp.n_stored + 1_000_000
    got, st = gpu_reasons(env, sp, w["Y"], 50, id_begin=b, id_end=e, precision=dse.PREC_FP64)
    check_equal(got, orc.reasons(b, e), st)
    sp.free()


@pytest.mark.parametrize("flags", [0, 4])
def test_reasons_tensor_core_targets(env, flags):
    """Sixteen targets on the multi-target Gram path (and, with
    DSE_FLAG_DIRECT, the sample-by-sample tensor-core kernel): the large
    workload's signed and lognormal primaries (domain masks fire), a 2e5-id
    slice of its pair block, and the precision primaries at rung 2."""
    torch, oracle, dse, W = env
    path = dse.PATH_TENSOR if flags else dse.PATH_GRAM_MT
    w = W.large(0, n_targets=16)
    sp, orc = spaces(env, w)
    # the unary block (sqrt and log of signed features fail their domain)
    # with the first pairs, then a slice deep in the pair block
    for b, e in ((sp.n_stored, sp.n_stored + 40_000), (sp.n_stored + 1_234_567, sp.n_stored + 1_434_567)):
        ref = orc.reasons(b, e)
        got, st = gpu_reasons(env, sp, w["Y"], 100, id_begin=b, id_end=e, precision=dse.PREC_AUTO, flags=flags)
        assert st["precision_used"] == dse.PREC_BF16X3
        assert st["binary_path"] == path
        check_equal(got, ref, st)
        assert np.sum(ref == 1) > 0 and np.sum(ref == 0) > 0
        if b == sp.n_stored:
            assert np.sum(ref == 3) > 0
    sp.free()
    w = dict(W.precision(0, n_targets=16), max_rung=2)
    sp, orc = spaces(env, w)
    got, st = gpu_reasons(env, sp, w["Y"], 100, precision=dse.PREC_AUTO, flags=flags)
    assert st["binary_path"] == path
    check_equal(got, orc.reasons(), st)
    sp.free()


@pytest.mark.parametrize("T", [2, 9])
def test_reasons_gram_multi_target_units(env, T):
    """The multi-target Gram path on the tiny workload, whose + and - are
    unit-checked (the kernel's own unit test of the sum and difference
    slots) and whose primaries are few enough for every candidate."""
    torch, oracle, dse, W = env
    for seed in (0, 1):
        w = W.tiny(seed)
        rng = np.random.default_rng(seed + 10 * T)
        Y = np.stack([w["Y"][0] + 0.3 * rng.standard_normal(w["X"].shape[1]) for _ in range(T)])
        sp, orc = spaces(env, w)
        got, st = gpu_reasons(env, sp, Y, 30, precision=dse.PREC_BF16X3)
        assert st["binary_path"] == dse.PATH_GRAM_MT
        ref = orc.reasons()
        check_equal(got, ref, st)
        assert np.sum(ref == 0) > 0
        sp.free()


@pytest.mark.parametrize("seed", [0, 1])
def test_reasons_extreme_scales(env, seed):
    """Features from 1e-12 to 1e12, mixed signs, a near-constant primary and
    every operator: magnitude masks fire and the FP32 kernels escalate to
    FP64; the realised decisions must still be the oracle's, one by one."""
    torch, oracle, dse, W = env
    from test_gpu_pairsum import ALL_OPS, stress_data

    X, y = stress_data(seed)
    sp = dse.Space(torch.from_numpy(X).cuda(), None, ALL_OPS, 2)
    orc = oracle.Space(X, None, ALL_OPS, 2)
    ref = orc.reasons()
    for prec in (dse.PREC_FP32, dse.PREC_FP64):
        got, st = gpu_reasons(env, sp, y[None, :], 50, precision=prec)
        check_equal(got, ref, st)
    assert np.sum(ref == 4) > 0 and np.sum(ref == 5) > 0
    sp.free()


@pytest.mark.parametrize("name", ["tiny", "medium", "large"])
def test_candidate_units(env, name):
    """Unit vectors of every stored feature and of 20000 seeded last-rung
    ids (all of them for tiny) against the oracle's, and the unit-valid flag
    against the oracle's unit rule."""
    torch, oracle, dse, W = env
    w = getattr(W, name)(0)
    sp, orc = spaces(env, w)
    rng = np.random.default_rng(5)
    last = np.arange(sp.n_stored, sp.n_total, dtype=np.uint64)
    if len(last) > 20000:
        last = np.sort(rng.choice(last, size=20000, replace=False))
    ids = np.concatenate([np.arange(sp.n_stored, dtype=np.uint64), last])
    units, ok = sp.candidate_units(ids)
    n_bad = 0
    for i, gid in enumerate(ids):
        ref = orc.candidate_unit(int(gid))
        if ref is None:
            assert ok[i] == 0, int(gid)
            n_bad += 1
        else:
            assert ok[i] == 1 and np.array_equal(units[i], ref), (int(gid), units[i], ref)
    assert n_bad > 0
    with pytest.raises(dse.DseError):
        sp.candidate_units(np.array([sp.n_total], np.uint64))
    sp.free()
