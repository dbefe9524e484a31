"""The score intervals of every screening path, before any re-score,
against the oracle's FP64 scores, candidate by candidate.

The returned top-k scores are re-scored, so they would stay within 1e-5 of
the oracle even if a kernel's bound were wrong; but which candidates reach
the buffers and which are certainly in or out of the top k is decided on the
kernels' own intervals [s - eps, s + eps].  For the tensor-core paths the
accumulation term of eps is a model of the MMA's rounding, not a proof.
Here every valid candidate of a sub-range gets its interval exported
(dse_screen_desc.intervals) and the oracle's score must lie inside it, for
every target: tensor-core BF16x3 with 16 targets (A operands in tensor
memory, N = 20000) and with 64 targets (A in shared memory, N = 500), the
product Gram contraction (one target, N = 1000), the sample-by-sample FP32
kernels (one and 16 targets) and the plain FP64 path.  Candidates without a
valid reason must have no interval, and valid ones one per target.
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


def spaces(env, w):
    torch, oracle, dse, W = env
    kw = dict(unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    sp = dse.Space(torch.from_numpy(w["X"]).cuda(), w["units"], w["op_mask"], w["max_rung"], **kw)
    orc = oracle.Space(w["X"], w["units"], w["op_mask"], w["max_rung"], **kw)
    return sp, orc


def check_intervals(env, sp, orc, Y, b, e, **kw):
    """Returns (number of candidate-target intervals checked, largest
    |s - oracle| / eps)."""
    torch = env[0]
    Y = np.ascontiguousarray(np.atleast_2d(Y))
    T, n = Y.shape[0], e - b
    ivl = torch.empty((n, T, 2), dtype=torch.float32, device="cuda")
    why = torch.empty(n, dtype=torch.int8, device="cuda")
    res = sp.screen(torch.from_numpy(Y).cuda(), 50, id_begin=b, id_end=e, reasons=why, intervals=ivl, **kw)
    res.stats()
    res.free()
    iv = ivl.cpu().numpy().astype(np.float64)
    valid = why.cpu().numpy() == 0
    has = ~np.isnan(iv[:, :, 0])
    assert np.array_equal(has.all(axis=1), valid) and np.array_equal(has.any(axis=1), valid)
    ids = np.arange(b, e, dtype=np.uint64)[valid]
    ref, rwhy = orc.score_ids(Y, ids)
    assert np.all(rwhy == 0)
    s, eps = iv[valid, :, 0], iv[valid, :, 1]
    assert np.all(eps >= 0)
    err = np.abs(s - ref)
    out = err > eps + 1e-12
    assert not out.any(), (f"{int(out.sum())} oracle scores outside their interval; worst "
                           f"|s - ref| = {err[out].max():.3e} against eps {eps[out][np.argmax(err[out])]:.3e}")
    return int(valid.sum()) * T, float(np.max(err / np.maximum(eps, 1e-300)))


@pytest.mark.parametrize("flags", [0, 4])
def test_intervals_tensor_core_16_targets(env, flags):
    """N = 20000, 16 targets: the multi-target Gram contraction (40 drained
    accumulation blocks) and, with DSE_FLAG_DIRECT, the sample-by-sample
    tensor-core kernel."""
    torch, oracle, dse, W = env
    w = W.large(0, n_targets=16)
    sp, orc = spaces(env, w)
    n_checked = 0
    # unary block and the first pairs; a slice deep in the pair block
    for b, e in ((sp.n_stored, sp.n_stored + 6000), (sp.n_stored + 3_456_789, sp.n_stored + 3_466_789)):
        n, worst = check_intervals(env, sp, orc, w["Y"], b, e, precision=dse.PREC_AUTO, flags=flags)
        n_checked += n
    assert n_checked > 50_000
    sp.free()


@pytest.mark.parametrize("T,N", [(2, 100), (7, 530), (16, 1000)])
def test_intervals_gram_multi_target(env, T, N):
    """The multi-target Gram contraction at a few target counts and sample
    counts: one accumulation block (N = 100), a ragged second block of one
    chunk (N = 530 = 16 chunks + 18 samples), two full blocks (N = 1000)."""
    torch, oracle, dse, W = env
    w = W.medium(3)
    w = dict(w, X=np.ascontiguousarray(w["X"][:, :N]))
    rng = np.random.default_rng(T * 1000 + N)
    X = w["X"]
    Y = np.stack([X[rng.integers(len(X))] * X[rng.integers(len(X))] / X[rng.integers(len(X))]
                  + 0.05 * rng.standard_normal(N) for _ in range(T)])
    sp, orc = spaces(env, w)
    b, e = sp.n_stored, min(sp.n_total, sp.n_stored + 60_000)
    n, worst = check_intervals(env, sp, orc, Y, b, e, precision=dse.PREC_BF16X3)
    assert n > 10_000
    sp.free()


def test_intervals_tensor_core_64_targets(env):
    torch, oracle, dse, W = env
    w = dict(W.precision(0, n_targets=64), max_rung=2)
    sp, orc = spaces(env, w)
    n, worst = check_intervals(env, sp, orc, w["Y"], sp.n_stored, min(sp.n_total, sp.n_stored + 40_000),
                               precision=dse.PREC_AUTO)
    assert n > 100_000
    sp.free()


@pytest.mark.parametrize("flags,precision", [(0, "fp32"), (4, "fp32"), (0, "fp64")])
def test_intervals_single_target(env, flags, precision):
    """Gram contraction of the products (flags 0, FP32), sample-by-sample
    FP32 (DSE_FLAG_DIRECT) and plain FP64 on the medium workload."""
    torch, oracle, dse, W = env
    w = W.medium(0)
    sp, orc = spaces(env, w)
    prec = dse.PREC_FP64 if precision == "fp64" else dse.PREC_FP32
    for b, e in ((0, sp.n_stored + 5000), (sp.n_stored + 700_000, sp.n_stored + 900_000)):
        check_intervals(env, sp, orc, w["Y"], b, e, precision=prec, flags=flags)
    sp.free()


def test_intervals_cuda_core_16_targets(env):
    """Sixteen targets on the CUDA-core FP32 kernels (16 targets a pass)."""
    torch, oracle, dse, W = env
    w = W.large(0, n_targets=16)
    sp, orc = spaces(env, w)
    check_intervals(env, sp, orc, w["Y"], sp.n_stored + 2_000_000, sp.n_stored + 2_006_000,
                    precision=dse.PREC_FP32)
    sp.free()
