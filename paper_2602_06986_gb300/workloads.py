"""Seeded synthetic inputs shaped like DISCOVER's materials-descriptor workloads.

This module only draws numbers: primary feature matrices, unit exponents,
planted targets and sample gather lists.  It holds none of the screening
arithmetic, so both the CUDA path and the CPU oracle take their inputs from it.
The application datasets the paper cites ("Scope and Use Cases") are not
available; these inputs stand in for them.

Every generator uses numpy's PCG64 with an explicit seed.  Values that a
workload declares as FP32 are drawn in FP64 and rounded to FP32, and the
rounded values (held as float64) are what both sides receive.

Op codes (bit positions of ``op_mask``): unary sq cb inv sqrt exp log = 0..5,
binary + - * a/b b/a |a-b| = 6..11.
"""
from __future__ import annotations

import numpy as np

SQUARE, CUBE, INV, SQRT, EXP, LOG, ADD, SUB, MUL, DIV, RDIV, ABSDIFF = range(12)


def mask(*codes):
    m = 0
    for c in codes:
        m |= 1 << c
    return m


#: + - * / (both slots) ^2 sqrt exp log
OPS_TINY = mask(ADD, SUB, MUL, DIV, RDIV, SQUARE, SQRT, EXP, LOG)
#: the full library: + - * / |-| ^2 ^3 ^-1 sqrt exp log
OPS_FULL = mask(*range(12))


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _units(rng, n0, dims):
    return rng.integers(-2, 3, size=(n0, dims)).astype(np.int32)


def tiny(seed: int = 0, noise: float = 0.01):
    """N=100, 8 primaries U[0.5,2] (FP64), units over 3 dims in -2..2; ops
    + - * / ^2 sqrt exp log; rung 2; only + and - are unit-checked; target
    2*x1*x3/x5^2 plus Gaussian noise of standard deviation ``noise``; top-100."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N, n0 = 100, 8
    X = rng.uniform(0.5, 2.0, size=(n0, N))
    units = _units(rng, n0, 3)
    y = 2.0 * X[1] * X[3] / X[5] ** 2 + noise * rng.standard_normal(N)
    return dict(name="tiny_n100_p8_rung2_top100", X=X, units=units, Y=y[None, :], op_mask=OPS_TINY,
                max_rung=2, unit_check_addsub=1, explog_dimensionless=0, k=100,
                planted="((x3*x1)/sq(x5))")


def medium(seed: int = 0):
    """N=1000, 20 primaries lognormal(0,0.5) (FP32), units over 4 dims; full op
    library; rung 2; full unit checks; planted two-term target c1*f_a + c2*f_b
    with f_a, f_b rung-2 products/quotients, plus 1% noise; top-1000 and the
    residual loop D = 1..3."""
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    N, n0 = 1000, 20
    X = _f32(rng.lognormal(0.0, 0.5, size=(n0, N)))
    units = _units(rng, n0, 4)
    p, q, r, s, t, u = rng.choice(n0, size=6, replace=False)
    fa = X[p] * X[q] / X[r] ** 2
    fb = (X[s] / X[t]) * np.sqrt(X[u])
    c1, c2 = 1.5, -0.8
    yc = c1 * fa + c2 * fb
    y = yc + 0.01 * yc.std() * rng.standard_normal(N)
    return dict(name="medium_n1000_p20_rung2_top1000_D3", X=X, units=units, Y=y[None, :], op_mask=OPS_FULL,
                max_rung=2, unit_check_addsub=1, explog_dimensionless=1, k=1000, D=3,
                planted_terms=(("mul_div_sq", int(p), int(q), int(r)), ("div_mul_sqrt", int(s), int(t), int(u))))


def _planted_targets(rng, X, T, noise_rel):
    n0, N = X.shape
    Y = np.empty((T, N))
    for t in range(T):
        a, b, c = rng.choice(n0, size=3, replace=False)
        kind = t % 4
        if kind == 0:
            f = X[a] * X[b] / X[c]
        elif kind == 1:
            f = (X[a] + X[b]) * X[c]
        elif kind == 2:
            f = np.sqrt(X[a]) * X[b] - X[c]
        else:
            f = X[a] / (X[b] + X[c])
        f = f + noise_rel * f.std() * rng.standard_normal(N)
        Y[t] = f
    return Y


def precision(seed: int = 0, n_targets: int = 64):
    """N=500, 12 primaries U[0.1,10] (FP32), dimensionless; full op library;
    rung 3 streamed in one block of 2^30 flat indices of the rung-3 binary
    block starting at a seeded offset; 64 planted targets with 1% noise;
    top-1000 per target."""
    rng = np.random.Generator(np.random.PCG64(3000 + seed))
    N, n0 = 500, 12
    X = _f32(rng.uniform(0.1, 10.0, size=(n0, N)))
    units = np.zeros((n0, 0), np.int32)
    Y = _planted_targets(rng, X, n_targets, 0.01)
    return dict(name="precision_n500_p12_rung3_block2e30_T64_top1000", X=X, units=units, Y=Y, op_mask=OPS_FULL,
                max_rung=3, unit_check_addsub=1, explog_dimensionless=1, k=1000,
                block_len=1 << 30, block_seed=int(rng.integers(0, 1 << 30)))


def large(seed: int = 0, n_targets: int = 16):
    """N=20000, 40 primaries: a third each U[0.5,5], lognormal(0,0.5) and
    N(0,1) (FP32), units over 5 dims; full op library; rung 2; 16 planted
    targets with 1% noise; top-10000 per target."""
    rng = np.random.Generator(np.random.PCG64(5000 + seed))
    N, n0 = 20000, 40
    parts = [rng.uniform(0.5, 5.0, size=(14, N)), rng.lognormal(0.0, 0.5, size=(13, N)),
             rng.standard_normal(size=(13, N))]
    X = _f32(np.concatenate(parts, axis=0))
    units = _units(rng, n0, 5)
    Y = _planted_targets(rng, np.abs(X) + 0.1, n_targets, 0.01)
    return dict(name="large_n20000_p40_rung2_T16_top10000", X=X, units=units, Y=Y, op_mask=OPS_FULL,
                max_rung=2, unit_check_addsub=1, explog_dimensionless=1, k=10000)


def batched(seed: int = 0, n_base: int = 32, n_folds: int = 5, n_boot: int = 3, n_hi: int = 5000,
            p_hi: int = 30):
    """256 problems = 32 base datasets x (5 CV-fold training sets + 3 bootstrap
    resamples).  Base sizes N_b are log-uniform so that problem sample counts
    span [50, 5000]; each base has 10-30 primaries U[0.5,5] (FP32) with units
    over 3 dims, the full op library, rung 2 and a planted target; top-200 per
    problem.  Each problem is (base index, sample gather list).  n_hi / p_hi
    shrink the largest base and primary count for cases the oracle screens
    in full."""
    rng = np.random.Generator(np.random.PCG64(4000 + seed))
    bases, problems = [], []
    lo, hi = np.log(50 / 0.8), np.log(n_hi)
    for b in range(n_base):
        Nb = int(round(np.exp(rng.uniform(lo, hi))))
        if b == 0:
            Nb = int(np.ceil(50 / 0.8))
        if b == 1:
            Nb = n_hi
        n0 = int(rng.integers(10, p_hi + 1))
        X = _f32(rng.uniform(0.5, 5.0, size=(n0, Nb)))
        units = _units(rng, n0, 3)
        a, c, d = rng.choice(n0, size=3, replace=False)
        yc = X[a] * X[c] / X[d]
        y = yc + 0.01 * yc.std() * rng.standard_normal(Nb)
        bases.append(dict(X=X, units=units, y=y))
        perm = rng.permutation(Nb)
        folds = np.array_split(perm, n_folds)
        for f in range(n_folds):
            train = np.sort(np.concatenate([folds[g] for g in range(n_folds) if g != f]))
            problems.append(dict(base=b, samples=train.astype(np.int64)))
        for _ in range(n_boot):
            problems.append(dict(base=b, samples=np.sort(rng.integers(0, Nb, size=Nb)).astype(np.int64)))
    return dict(name="batched_256problems_n50to5000_p10to30_rung2_top200", bases=bases, problems=problems,
                op_mask=OPS_FULL, max_rung=2, unit_check_addsub=1, explog_dimensionless=1, k=200)
