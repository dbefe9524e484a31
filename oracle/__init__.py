"""Plain FP64 CPU oracle for SIS screening of a SISSO-style feature space.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
and its Python binding never import, link or call anything here, and the two
share no code.

The arithmetic lives in ``oracle.c`` (IEEE FP64, OpenMP over candidates).  This
module is argument marshalling over it with ``ctypes`` plus two small pure
Python references used to pin it: ``enumerate_bruteforce`` (expression trees
built recursively with exact ``fractions.Fraction`` unit exponents) and the
closed-form counters in ``counts.py``.

Op codes (the slot order of a pair, and the bits of ``op_mask``):
unary ``sq cb inv sqrt exp log`` = 0..5, binary ``+ - * a/b b/a |a-b|`` = 6..11.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SRC_PATH = os.path.join(HERE, "oracle.c")

SQUARE, CUBE, INV, SQRT, EXP, LOG, ADD, SUB, MUL, DIV, RDIV, ABSDIFF = range(12)
PRIMARY = 15
OP_NAMES = ["sq", "cb", "inv", "sqrt", "exp", "log", "+", "-", "*", "a/b", "b/a", "|a-b|"]
REASONS = ["valid", "unit", "complexity", "domain", "magnitude", "realised"]
# reason 2 also counts candidates failing a variable-combination or
# functional-form rule (the "form" reason: complexity cap or rule)


def op_mask(*codes):
    m = 0
    for c in codes:
        m |= 1 << c
    return m


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, FP64, no FMA contraction)."""
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC_PATH)):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
           "-shared", "-fPIC", SRC_PATH, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Params(C.Structure):
    _fields_ = [
        ("n_samples", C.c_int64), ("n_primary", C.c_int64),
        ("n_dims", C.c_int32), ("max_rung", C.c_int32),
        ("X", C.POINTER(C.c_double)), ("units", C.POINTER(C.c_int32)),
        ("op_mask", C.c_uint32), ("max_complexity", C.c_int32),
        ("unit_check_addsub", C.c_int32), ("explog_dimensionless", C.c_int32),
        ("fmax_max", C.c_double), ("fmin_std_rel", C.c_double),
        ("pair_deny", C.POINTER(C.c_uint64)), ("op_deny", C.POINTER(C.c_uint64)),
    ]


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB_PATH)
            vp, i64, u64, i32, dp = C.c_void_p, C.c_int64, C.c_uint64, C.c_int32, C.POINTER(C.c_double)
            L.orc_space_build.argtypes = [C.POINTER(_Params), C.POINTER(vp)]
            L.orc_space_build.restype = C.c_int
            L.orc_space_free.argtypes = [vp]
            L.orc_n_features.argtypes = [vp]; L.orc_n_features.restype = i64
            L.orc_rung_begin.argtypes = [vp, C.c_int]; L.orc_rung_begin.restype = i64
            L.orc_rung_slots.argtypes = [vp, C.c_int]; L.orc_rung_slots.restype = u64
            L.orc_total_candidates.argtypes = [vp]; L.orc_total_candidates.restype = u64
            L.orc_rung_counts.argtypes = [vp, C.c_int, C.POINTER(i64), C.POINTER(i64)]
            L.orc_decode.argtypes = [vp, u64, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64), C.POINTER(i64)]
            L.orc_expr_string.argtypes = [vp, u64, C.c_char_p, i64]
            L.orc_candidate.argtypes = [vp, u64, dp, C.POINTER(i32)]
            L.orc_feature_info.argtypes = [vp, i64, C.POINTER(i32), C.POINTER(i64), dp]
            L.orc_screen.argtypes = [vp, dp, C.c_int, i64, C.c_int, u64, u64,
                                     C.POINTER(u64), dp, C.POINTER(i64), C.POINTER(i64)]
            L.orc_score_ids.argtypes = [vp, dp, C.c_int, C.POINTER(u64), i64, dp, C.POINTER(i32)]
            L.orc_residual_loop.argtypes = [vp, dp, C.c_int, i64, C.POINTER(u64), dp, dp,
                                            C.POINTER(u64), C.POINTER(i64), dp]
            L.orc_num_threads.restype = C.c_int
            L.orc_margins.argtypes = [vp, C.c_int, u64, u64, dp]
            L.orc_margins.restype = C.c_int
            L.orc_l0_search.argtypes = [vp, dp, C.POINTER(u64), i64, C.c_int, i64, C.POINTER(i64), dp,
                                        C.POINTER(i64)]
            L.orc_l0_search.restype = C.c_int
            L.orc_screen_dedup.argtypes = [vp, dp, C.c_int, i64, C.c_int, C.c_double, u64, u64, C.POINTER(u64),
                                           dp, C.POINTER(i64), C.POINTER(i64), dp]
            L.orc_screen_dedup.restype = C.c_int
            L.orc_reasons.argtypes = [vp, u64, u64, C.POINTER(C.c_int8)]
            L.orc_reasons.restype = C.c_int
            L.orc_candidate_unit.argtypes = [vp, u64, C.POINTER(i64)]
            L.orc_candidate_unit.restype = C.c_int
            _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def num_threads() -> int:
    return int(lib().orc_num_threads())


class Space:
    """Phi_{k-1} materialised in FP64 plus the enumeration of rung k.

    ``X`` is ``[n_primary, n_samples]`` float64, ``units`` ``[n_primary, n_dims]``
    int32 exponents.  Global candidate ids: ``[0, n_features)`` are the stored
    features of rungs < max_rung, ``n_features + p`` is flat index ``p`` of
    rung ``max_rung``.
    """

    def __init__(self, X, units, op_mask, max_rung, max_complexity=0, unit_check_addsub=1,
                 explog_dimensionless=1, fmax_max=1e15, fmin_std_rel=1e-8, pair_deny=None, op_deny=None):
        """``pair_deny`` (uint64 [n_primary]: bit q of row p forbids primaries
        p and q in one expression) and ``op_deny`` (uint64 [12]: bit p of row o
        forbids primary p below op o) are the optional user rules of R15."""
        L = lib()
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        n_primary, n_samples = self.X.shape
        units = np.zeros((n_primary, 0), np.int32) if units is None else units
        self.units = np.ascontiguousarray(units, dtype=np.int32)
        assert self.units.shape[0] == n_primary
        u64p = C.POINTER(C.c_uint64)
        self._pd = None if pair_deny is None else np.ascontiguousarray(pair_deny, dtype=np.uint64)
        self._od = None if op_deny is None else np.ascontiguousarray(op_deny, dtype=np.uint64)
        assert self._pd is None or self._pd.shape == (n_primary,)
        assert self._od is None or self._od.shape == (12,)
        p = _Params(n_samples, n_primary, self.units.shape[1], max_rung, _dptr(self.X),
                    self.units.ctypes.data_as(C.POINTER(C.c_int32)), op_mask, max_complexity,
                    unit_check_addsub, explog_dimensionless, fmax_max, fmin_std_rel,
                    None if self._pd is None else self._pd.ctypes.data_as(u64p),
                    None if self._od is None else self._od.ctypes.data_as(u64p))
        h = C.c_void_p()
        rc = L.orc_space_build(C.byref(p), C.byref(h))
        if rc != 0:
            raise ValueError(f"orc_space_build failed: {rc}")
        self._h = h
        self.n_samples = n_samples
        self.max_rung = max_rung
        self.n_dims = self.units.shape[1]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_space_free(h)
            self._h = None

    @property
    def n_features(self) -> int:
        return int(lib().orc_n_features(self._h))

    def rung_begin(self, r: int) -> int:
        return int(lib().orc_rung_begin(self._h, r))

    def rung_slots(self, r: int) -> int:
        return int(lib().orc_rung_slots(self._h, r))

    @property
    def total_candidates(self) -> int:
        return int(lib().orc_total_candidates(self._h))

    def rung_counts(self, r: int):
        """(slots, {reason: count}) of rung r; rung max_rung is evaluated in full."""
        slots = C.c_int64()
        rs = (C.c_int64 * 6)()
        rc = lib().orc_rung_counts(self._h, r, C.byref(slots), rs)
        if rc:
            raise ValueError(rc)
        return int(slots.value), {REASONS[i]: int(rs[i]) for i in range(6)}

    def decode(self, gid: int):
        """Global id -> (rung, op, a, b); for a stored rung-0 feature a is the primary index."""
        r, op = C.c_int32(), C.c_int32()
        a, b = C.c_int64(), C.c_int64()
        if lib().orc_decode(self._h, gid, C.byref(r), C.byref(op), C.byref(a), C.byref(b)):
            raise IndexError(gid)
        return r.value, op.value, a.value, b.value

    def expr(self, gid: int) -> str:
        buf = C.create_string_buffer(1 << 14)
        if lib().orc_expr_string(self._h, gid, buf, len(buf)):
            raise IndexError(gid)
        return buf.value.decode()

    def candidate(self, gid: int):
        """(values float64[N] or None, reason code)."""
        v = np.zeros(self.n_samples)
        why = C.c_int32()
        if lib().orc_candidate(self._h, gid, _dptr(v), C.byref(why)):
            raise IndexError(gid)
        return (v if why.value == 0 else None), why.value

    def reasons(self, id_begin: int = 0, id_end=None):
        """Reason code (int8, 0 = valid) of every candidate id in [id_begin, id_end)."""
        id_end = self.total_candidates if id_end is None else id_end
        out = np.zeros(max(id_end - id_begin, 0), np.int8)
        if lib().orc_reasons(self._h, id_begin, id_end, out.ctypes.data_as(C.POINTER(C.c_int8))):
            raise IndexError((id_begin, id_end))
        return out

    def candidate_unit(self, gid: int):
        """(unit exponents int64[n_dims] scaled by 2^max_rung, or None when
        the op's unit rule fails)."""
        u = np.zeros(max(self.n_dims, 1), np.int64)
        rc = lib().orc_candidate_unit(self._h, gid, u.ctypes.data_as(C.POINTER(C.c_int64)))
        if rc < 0:
            raise IndexError(gid)
        return u[: self.n_dims].copy() if rc == 1 else None

    def feature_info(self, f: int):
        cx = C.c_int32()
        u = np.zeros(max(self.n_dims, 1), np.int64)
        s4 = np.zeros(4)
        if lib().orc_feature_info(self._h, f, C.byref(cx), u.ctypes.data_as(C.POINTER(C.c_int64)), _dptr(s4)):
            raise IndexError(f)
        return {"complexity": cx.value, "unit": u[: self.n_dims].copy(), "min": s4[0], "max": s4[1],
                "minabs": s4[2], "maxabs": s4[3]}

    def screen(self, Y, k: int, mode: str = "per_target", id_begin: int = 0, id_end=None):
        """Top-k by SIS score.  Returns (ids list-of-arrays, scores list-of-arrays, counts)."""
        Y = np.ascontiguousarray(np.atleast_2d(Y), dtype=np.float64)
        T = Y.shape[0]
        assert Y.shape[1] == self.n_samples
        m = {"per_target": 0, "aggregated": 1}[mode]
        Lc = T if m == 0 else 1
        if id_end is None:
            id_end = self.total_candidates
        ids = np.zeros((Lc, k), np.uint64)
        sc = np.zeros((Lc, k))
        n = np.zeros(Lc, np.int64)
        cnt = np.zeros(6, np.int64)
        rc = lib().orc_screen(self._h, _dptr(Y), T, k, m, id_begin, id_end,
                              ids.ctypes.data_as(C.POINTER(C.c_uint64)), _dptr(sc),
                              n.ctypes.data_as(C.POINTER(C.c_int64)), cnt.ctypes.data_as(C.POINTER(C.c_int64)))
        if rc:
            raise ValueError(f"orc_screen failed: {rc}")
        return ([ids[l, : n[l]].copy() for l in range(Lc)], [sc[l, : n[l]].copy() for l in range(Lc)],
                {REASONS[i]: int(cnt[i]) for i in range(6)})

    def screen_dedup(self, Y, k: int, tau: float = 1e-10, mode: str = "per_target", id_begin: int = 0,
                     id_end=None):
        """Top-k of the non-redundant candidates (R16).  Returns (ids per list,
        scores per list, redundant entries passed over per list, smallest
        correlation margin | (1 - |rho|) - tau |)."""
        Y = np.ascontiguousarray(np.atleast_2d(Y), dtype=np.float64)
        T = Y.shape[0]
        m = {"per_target": 0, "aggregated": 1}[mode]
        Lc = T if m == 0 else 1
        if id_end is None:
            id_end = self.total_candidates
        ids = np.zeros((Lc, k), np.uint64)
        sc = np.zeros((Lc, k))
        n = np.zeros(Lc, np.int64)
        red = np.zeros(Lc, np.int64)
        mg = C.c_double()
        rc = lib().orc_screen_dedup(self._h, _dptr(Y), T, k, m, tau, id_begin, id_end,
                                    ids.ctypes.data_as(C.POINTER(C.c_uint64)), _dptr(sc),
                                    n.ctypes.data_as(C.POINTER(C.c_int64)), red.ctypes.data_as(C.POINTER(C.c_int64)),
                                    C.byref(mg))
        if rc:
            raise ValueError(f"orc_screen_dedup failed: {rc}")
        return ([ids[l, : n[l]].copy() for l in range(Lc)], [sc[l, : n[l]].copy() for l in range(Lc)],
                red.copy(), mg.value)

    def score_ids(self, Y, ids):
        """(scores [n, T] with NaN for invalid ids, reason codes [n])."""
        Y = np.ascontiguousarray(np.atleast_2d(Y), dtype=np.float64)
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        T = Y.shape[0]
        sc = np.zeros((len(ids), T))
        why = np.zeros(len(ids), np.int32)
        if lib().orc_score_ids(self._h, _dptr(Y), T, ids.ctypes.data_as(C.POINTER(C.c_uint64)), len(ids),
                               _dptr(sc), why.ctypes.data_as(C.POINTER(C.c_int32))):
            raise ValueError("orc_score_ids failed")
        return sc, why

    def l0_search(self, y, ids, D: int, m_top: int = 16):
        """Exhaustive search of the best D-subsets of the listed candidates
        (Eq. 1 over a subspace): (positions int64[m, D], RMSE[m]) in the order
        (RMSE ascending, positions lexicographically ascending)."""
        y = np.ascontiguousarray(y, dtype=np.float64)
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        pos = np.zeros((m_top, D), np.int64)
        rm = np.zeros(m_top)
        nf = C.c_int64()
        if lib().orc_l0_search(self._h, _dptr(y), ids.ctypes.data_as(C.POINTER(C.c_uint64)), len(ids), D, m_top,
                               pos.ctypes.data_as(C.POINTER(C.c_int64)), _dptr(rm), C.byref(nf)):
            raise ValueError("orc_l0_search failed")
        return pos[:nf.value].copy(), rm[:nf.value].copy()

    def margins(self, rung: int, p_begin: int = 0, p_end=None):
        """Smallest relative margins of the magnitude, exp-domain and realised
        tests over flat slots [p_begin, p_end) of ``rung`` (and the slot count)."""
        out = np.zeros(4)
        if p_end is None:
            p_end = np.iinfo(np.uint64).max
        if lib().orc_margins(self._h, rung, p_begin, p_end, _dptr(out)):
            raise ValueError("orc_margins failed")
        return {"magnitude": out[0], "exp_domain": out[1], "realised": out[2], "slots": int(out[3])}

    def residual_loop(self, y, Dmax: int, k: int):
        y = np.ascontiguousarray(y, dtype=np.float64)
        desc = np.zeros(Dmax, np.uint64)
        rmse = np.zeros(Dmax)
        coefs = np.zeros((Dmax, Dmax + 1))
        sis = np.zeros((Dmax, k), np.uint64)
        nsis = np.zeros(Dmax, np.int64)
        res = np.zeros(self.n_samples)
        rc = lib().orc_residual_loop(self._h, _dptr(y), Dmax, k, desc.ctypes.data_as(C.POINTER(C.c_uint64)),
                                     _dptr(rmse), _dptr(coefs), sis.ctypes.data_as(C.POINTER(C.c_uint64)),
                                     nsis.ctypes.data_as(C.POINTER(C.c_int64)), _dptr(res))
        if rc:
            raise ValueError(f"orc_residual_loop failed: {rc}")
        return {"ids": desc, "rmse": rmse, "coefs": coefs,
                "sis": [sis[d, : nsis[d]].copy() for d in range(Dmax)], "residual": res}
