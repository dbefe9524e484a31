"""Python binding of libdse.so: argument marshalling over the C ABI (include/dse.h).

Every computation runs in the CUDA library; this module only packs
descriptors, passes pointers (numpy arrays for host memory, ``torch`` tensors'
``data_ptr()`` for device memory) and raises ``DseError`` on a non-zero
status.  Importing it loads the in-tree library and fails loudly if it is
missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
# DSE_LIB_VARIANT=checked loads the bounds-checked build (DSE_CHECK_BOUNDS)
LIB_PATH = os.path.join(PKG, "libdse_checked.so" if os.environ.get("DSE_LIB_VARIANT") == "checked" else "libdse.so")

OK, EINVAL, ENOMEM, ECUDA, ERANGE, ETIMEOUT, EOVERFLOW, EBOUNDS = 0, -1, -2, -3, -4, -5, -6, -7
SQUARE, CUBE, INV, SQRT, EXP, LOG, ADD, SUB, MUL, DIV, RDIV, ABSDIFF = range(12)
PRIMARY = 15
MODE_PER_TARGET, MODE_AGGREGATED = 0, 1
PREC_FP32, PREC_FP64, PREC_BF16X3, PREC_AUTO = 0, 1, 2, 3
REASONS = ["valid", "unit", "complexity", "domain", "magnitude", "realised"]


class DseError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"dse status {status}: {msg}")
        self.status = status


class SpaceDesc(C.Structure):
    _fields_ = [("n_samples", C.c_int64), ("n_primary", C.c_int64), ("n_dims", C.c_int32),
                ("max_rung", C.c_int32), ("X", C.c_void_p), ("ld_x", C.c_int64), ("x_on_device", C.c_int32),
                ("reserved0", C.c_int32), ("sample_idx", C.c_void_p), ("units", C.c_void_p),
                ("op_mask", C.c_uint32), ("max_complexity", C.c_int32), ("unit_check_addsub", C.c_int32),
                ("explog_dimensionless", C.c_int32), ("fmax_max", C.c_double), ("fmin_std_rel", C.c_double),
                ("stream", C.c_void_p), ("pair_deny", C.c_void_p), ("op_deny", C.c_void_p)]


class ScreenDesc(C.Structure):
    _fields_ = [("Y", C.c_void_p), ("ld_y", C.c_int64), ("y_on_device", C.c_int32), ("n_targets", C.c_int32),
                ("k", C.c_int64), ("mode", C.c_int32), ("precision", C.c_int32), ("id_begin", C.c_uint64),
                ("id_end", C.c_uint64), ("stream", C.c_void_p), ("flags", C.c_int32), ("reserved0", C.c_int32),
                ("dedup_tau", C.c_double), ("reasons", C.c_void_p), ("intervals", C.c_void_p)]


class Tuning(C.Structure):
    _fields_ = [("tile_group", C.c_int32), ("seed_stride", C.c_int32), ("gram_max_n", C.c_int32),
                ("tc_min_targets", C.c_int32), ("batch_job_samples", C.c_int32), ("gmt_group", C.c_int32),
                ("gmt_cluster", C.c_int32), ("reserved", C.c_int32 * 1)]


TUNING_FIELDS = ("tile_group", "seed_stride", "gram_max_n", "tc_min_targets", "batch_job_samples", "gmt_group",
                 "gmt_cluster")

FLAG_TIMING = 1
FLAG_DEDUP = 2
FLAG_DIRECT = 4
FLAG_TIMING_MAIN = 8
# dse_stats.binary_path
PATH_CUDA_CORE, PATH_TENSOR, PATH_GRAM, PATH_GRAM_MT = 1, 2, 3, 4


class Stats(C.Structure):
    _fields_ = [("screened", C.c_int64), ("reasons", C.c_int64 * 6), ("evaluated", C.c_int64),
                ("buffered", C.c_int64), ("escalated", C.c_int64), ("rescored", C.c_int64),
                ("reruns", C.c_int32), ("precision_used", C.c_int32), ("max_err_bound", C.c_double),
                ("valid_by_group", C.c_int64 * 3), ("kernel_ms", C.c_double * 4), ("kernel_launches", C.c_int64),
                ("redundant", C.c_int64), ("dedup_rounds", C.c_int32), ("binary_path", C.c_int32)]


class Expr(C.Structure):
    _fields_ = [("rung", C.c_int32), ("op", C.c_int32), ("a", C.c_int64), ("b", C.c_int64)]


class RefitDesc(C.Structure):
    _fields_ = [("y", C.c_void_p), ("y_on_device", C.c_int32), ("n_fixed", C.c_int32), ("fixed", C.c_void_p),
                ("cand", C.c_void_p), ("n_cand", C.c_int64), ("cand_on_device", C.c_int32),
                ("reserved0", C.c_int32), ("stream", C.c_void_p)]


class BatchItem(C.Structure):
    _fields_ = [("space", C.c_void_p), ("y", C.c_void_p), ("y_on_device", C.c_int32), ("reserved0", C.c_int32)]


class BatchDesc(C.Structure):
    _fields_ = [("k", C.c_int64), ("precision", C.c_int32), ("flags", C.c_int32), ("stream", C.c_void_p)]


BATCH_GRAPH = 1


class LoopDesc(C.Structure):
    _fields_ = [("y", C.c_void_p), ("y_on_device", C.c_int32), ("n_iter", C.c_int32), ("k", C.c_int64),
                ("precision", C.c_int32), ("flags", C.c_int32), ("stream", C.c_void_p), ("n_fixed", C.c_int32),
                ("reserved0", C.c_int32), ("fixed", C.c_void_p)]


class L0Desc(C.Structure):
    _fields_ = [("y", C.c_void_p), ("y_on_device", C.c_int32), ("dim", C.c_int32), ("ids", C.c_void_p),
                ("n_ids", C.c_int64), ("ids_on_device", C.c_int32), ("n_top", C.c_int32), ("stream", C.c_void_p)]


class LoopResult(C.Structure):
    _fields_ = [("chosen", C.c_uint64 * 4), ("rmse", C.c_double * 4), ("coefs", (C.c_double * 5) * 4),
                ("stats", Stats * 4)]

EXPORTS = ["dse_build_space", "dse_space_free", "dse_space_size", "dse_space_counts", "dse_decode",
           "dse_expr_string", "dse_candidate_units", "dse_sis_screen", "dse_result_free", "dse_topk_fetch", "dse_result_stats",
           "dse_sis_screen_batched", "dse_batch_rescreen", "dse_batch_fetch", "dse_batch_stats", "dse_batch_free",
           "dse_residual_loop", "dse_l0_search", "dse_ls_refit", "dse_ls_refit_noalloc", "dse_check_wait",
           "dse_measure_peaks", "dse_bounds_probe",
           "dse_debug_fail_alloc", "dse_set_tuning", "dse_get_tuning", "dse_kernel_launches", "dse_last_error",
           "dse_version"]

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
        L.dse_build_space.argtypes = [C.POINTER(SpaceDesc), C.POINTER(vp)]
        L.dse_space_free.argtypes = [vp]
        L.dse_space_free.restype = None
        L.dse_space_size.argtypes = [vp, C.POINTER(i64), C.POINTER(u64)]
        L.dse_space_counts.argtypes = [vp, i32, C.POINTER(u64), C.POINTER(i64)]
        L.dse_decode.argtypes = [vp, u64, C.POINTER(Expr)]
        L.dse_expr_string.argtypes = [vp, u64, C.c_char_p, i64]
        L.dse_candidate_units.argtypes = [vp, vp, i64, vp, vp]
        L.dse_sis_screen.argtypes = [vp, C.POINTER(ScreenDesc), C.POINTER(vp)]
        L.dse_result_free.argtypes = [vp]
        L.dse_result_free.restype = None
        L.dse_topk_fetch.argtypes = [vp, i32, vp, vp, vp, i64, C.POINTER(i64)]
        L.dse_result_stats.argtypes = [vp, C.POINTER(Stats)]
        L.dse_sis_screen_batched.argtypes = [C.POINTER(BatchItem), i32, C.POINTER(BatchDesc), C.POINTER(vp)]
        L.dse_batch_rescreen.argtypes = [vp, vp, i32]
        L.dse_batch_fetch.argtypes = [vp, i32, vp, vp, vp, i64, C.POINTER(i64)]
        L.dse_batch_stats.argtypes = [vp, i32, C.POINTER(Stats)]
        L.dse_batch_free.argtypes = [vp]
        L.dse_batch_free.restype = None
        L.dse_residual_loop.argtypes = [vp, C.POINTER(LoopDesc), C.POINTER(LoopResult), vp, vp]
        L.dse_l0_search.argtypes = [vp, C.POINTER(L0Desc), vp, vp, vp, C.POINTER(i32)]
        L.dse_ls_refit.argtypes = [vp, C.POINTER(RefitDesc), C.POINTER(u64), C.POINTER(C.c_double), vp, vp]
        L.dse_ls_refit_noalloc.argtypes = L.dse_ls_refit.argtypes
        L.dse_check_wait.argtypes = [C.c_uint32, i32, vp]
        L.dse_measure_peaks.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
        L.dse_bounds_probe.argtypes = [i64, i64, vp]
        L.dse_set_tuning.argtypes = [C.POINTER(Tuning)]
        L.dse_get_tuning.argtypes = [C.POINTER(Tuning)]
        L.dse_debug_fail_alloc.argtypes = [i64]
        L.dse_debug_fail_alloc.restype = None
        L.dse_last_error.restype = C.c_char_p
        L.dse_version.restype = C.c_char_p
        L.dse_kernel_launches.restype = i64
        for name in EXPORTS:
            if name not in ("dse_space_free", "dse_result_free", "dse_batch_free", "dse_last_error",
                            "dse_version", "dse_kernel_launches", "dse_debug_fail_alloc"):
                getattr(L, name).restype = i32
        _lib = L
    return _lib


def set_tuning(values=None):
    """Install planner parameters (dse_set_tuning): a dict with any of
    TUNING_FIELDS (missing or 0: default); None restores every default."""
    if values is None:
        _check(lib().dse_set_tuning(None))
        return
    unknown = set(values) - set(TUNING_FIELDS)
    if unknown:
        raise ValueError(f"unknown tuning fields {sorted(unknown)}")
    t = Tuning(*(int(values.get(f, 0)) for f in TUNING_FIELDS))
    _check(lib().dse_set_tuning(C.byref(t)))


def get_tuning():
    """The planner parameters in effect (dse_get_tuning)."""
    t = Tuning()
    _check(lib().dse_get_tuning(C.byref(t)))
    return {f: getattr(t, f) for f in TUNING_FIELDS}


def check_wait(polls, arrive, stream=None):
    """Status of the bounded device wait probe (dse_check_wait)."""
    return int(lib().dse_check_wait(polls, 1 if arrive else 0, stream))


def measure_peaks(stream=None) -> dict:
    """Issue rates of the FP32 FMA, MUFU and FP64 FMA pipes on the current
    device, lane operations per second (dse_measure_peaks)."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(lib().dse_measure_peaks(C.byref(a), C.byref(b), C.byref(c), stream))
    return {"fp32_fma_per_s": a.value, "sfu_per_s": b.value, "fp64_fma_per_s": c.value}


def bounds_probe(index, limit, stream=None):
    """Status of one device-side index check (dse_bounds_probe): EBOUNDS
    outside [0, limit), OK inside; EINVAL in a build without the checks."""
    return int(lib().dse_bounds_probe(index, limit, stream))


def debug_fail_alloc(after):
    """Make the device allocation after ``after`` more successful ones fail
    with DSE_ENOMEM (negative: off)."""
    lib().dse_debug_fail_alloc(after)


def _check(status):
    if status != OK:
        raise DseError(status, lib().dse_last_error().decode())


def _ptr(a):
    """(pointer, on_device) of a numpy array or a torch tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError(type(a))


def version() -> str:
    return lib().dse_version().decode()


class Result:
    """A screen's result handle (device resident until fetched)."""

    def __init__(self, handle, n_lists, k):
        self._h = handle
        self.n_lists = n_lists
        self.k = k

    def fetch(self, lst=0, out=None):
        """(ids uint64, scores float64, err_bounds float64) of list ``lst``.
        With ``out`` = (ids, scores, bounds) torch CUDA tensors the copy stays on
        the device and the return value is the list length."""
        n = C.c_int64()
        if out is not None:
            pi, ps, pe = (t.data_ptr() for t in out)
            _check(lib().dse_topk_fetch(self._h, lst, pi, ps, pe, out[0].numel(), C.byref(n)))
            return n.value
        ids = np.zeros(self.k, np.uint64)
        sc = np.zeros(self.k)
        eb = np.zeros(self.k)
        _check(lib().dse_topk_fetch(self._h, lst, ids.ctypes.data, sc.ctypes.data, eb.ctypes.data, self.k,
                                    C.byref(n)))
        m = n.value
        return ids[:m].copy(), sc[:m].copy(), eb[:m].copy()

    def stats(self) -> dict:
        s = Stats()
        _check(lib().dse_result_stats(self._h, C.byref(s)))
        return _stats_dict(s)

    def free(self):
        if self._h:
            lib().dse_result_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _stats_dict(s) -> dict:
    return {"screened": s.screened, "reasons": {REASONS[i]: s.reasons[i] for i in range(6)},
                "evaluated": s.evaluated, "buffered": s.buffered, "escalated": s.escalated,
                "rescored": s.rescored, "reruns": s.reruns, "precision_used": s.precision_used,
                "max_err_bound": s.max_err_bound, "valid_by_group": list(s.valid_by_group),
            "kernel_ms": list(s.kernel_ms), "kernel_launches": s.kernel_launches,
            "redundant": s.redundant, "dedup_rounds": s.dedup_rounds, "binary_path": s.binary_path}


class Batch:
    """A batched screen over many (space, target) problems (dse_sis_screen_batched).

    ``spaces``: Space objects (kept alive by the batch); ``targets``: one
    target per space (numpy arrays or torch CUDA tensors of that space's
    n_samples values).  The first screen is enqueued at construction;
    ``rescreen`` screens again with new targets (replaying a CUDA graph with
    ``graph=True``)."""

    def __init__(self, spaces, targets, k, precision=PREC_FP32, graph=False, stream=None):
        self.spaces = list(spaces)
        self.k = k
        self._keep = []
        items = (BatchItem * len(self.spaces))()
        for i, (sp, y) in enumerate(zip(self.spaces, targets)):
            if isinstance(y, np.ndarray):
                y = np.ascontiguousarray(y, dtype=np.float64)
            self._keep.append(y)
            py, ydev = _ptr(y)
            items[i] = BatchItem(sp._h.value, py, ydev, 0)
        d = BatchDesc(k, precision, BATCH_GRAPH if graph else 0, stream)
        h = C.c_void_p()
        _check(lib().dse_sis_screen_batched(items, len(self.spaces), C.byref(d), C.byref(h)))
        self._h = h

    def rescreen(self, Ycat):
        """New targets, concatenated in problem order."""
        if isinstance(Ycat, np.ndarray):
            Ycat = np.ascontiguousarray(Ycat, dtype=np.float64)
        self._ycat = Ycat
        py, ydev = _ptr(Ycat)
        _check(lib().dse_batch_rescreen(self._h, py, ydev))

    def fetch(self, item):
        n = C.c_int64()
        ids = np.zeros(self.k, np.uint64)
        sc = np.zeros(self.k)
        eb = np.zeros(self.k)
        _check(lib().dse_batch_fetch(self._h, item, ids.ctypes.data, sc.ctypes.data, eb.ctypes.data, self.k,
                                     C.byref(n)))
        m = n.value
        return ids[:m].copy(), sc[:m].copy(), eb[:m].copy()

    def stats(self, item) -> dict:
        s = Stats()
        _check(lib().dse_batch_stats(self._h, item, C.byref(s)))
        return _stats_dict(s)

    def free(self):
        if getattr(self, "_h", None):
            lib().dse_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Space:
    """A built feature space (device resident)."""

    def __init__(self, X, units, op_mask, max_rung, max_complexity=0, unit_check_addsub=1, explog_dimensionless=1,
                 fmax_max=1e15, fmin_std_rel=1e-8, sample_idx=None, stream=None, pair_deny=None, op_deny=None):
        """pair_deny: uint64 [n_primary] rows (bit q of row p: primaries p and q
        never in one expression; bit p of row p: p at most once); op_deny:
        uint64 [12] rows by op code (bit p: primary p never below that op)."""
        self._keep = []
        if pair_deny is not None:
            pair_deny = np.ascontiguousarray(pair_deny, dtype=np.uint64)
            if pair_deny.shape != (X.shape[0],):
                raise ValueError("pair_deny must have one uint64 row per primary")
        if op_deny is not None:
            op_deny = np.ascontiguousarray(op_deny, dtype=np.uint64)
            if op_deny.shape != (12,):
                raise ValueError("op_deny must have 12 uint64 rows")
        self._keep += [pair_deny, op_deny]
        if isinstance(X, np.ndarray):
            X = np.ascontiguousarray(X, dtype=np.float64)
        n_primary, ld = X.shape
        if units is None:
            units = np.zeros((n_primary, 0), np.int32)
        units = np.ascontiguousarray(units, dtype=np.int32)
        n_samples = ld if sample_idx is None else len(sample_idx)
        if sample_idx is not None:
            sample_idx = np.ascontiguousarray(sample_idx, dtype=np.int64)
        self._keep += [X, units, sample_idx]
        px, xdev = _ptr(X)
        d = SpaceDesc(n_samples, n_primary, units.shape[1], max_rung, px, ld, xdev, 0,
                      sample_idx.ctypes.data if sample_idx is not None else None,
                      units.ctypes.data if units.shape[1] else None, op_mask, max_complexity, unit_check_addsub,
                      explog_dimensionless, fmax_max, fmin_std_rel, stream,
                      pair_deny.ctypes.data if pair_deny is not None else None,
                      op_deny.ctypes.data if op_deny is not None else None)
        h = C.c_void_p()
        _check(lib().dse_build_space(C.byref(d), C.byref(h)))
        self._h = h
        self.n_samples = n_samples
        self.max_rung = max_rung
        self.n_dims = units.shape[1]
        ns, nt = C.c_int64(), C.c_uint64()
        _check(lib().dse_space_size(self._h, C.byref(ns), C.byref(nt)))
        self.n_stored, self.n_total = ns.value, nt.value

    def free(self):
        if getattr(self, "_h", None):
            lib().dse_space_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def counts(self, rung):
        slots = C.c_uint64()
        r = (C.c_int64 * 6)()
        _check(lib().dse_space_counts(self._h, rung, C.byref(slots), r))
        return int(slots.value), {REASONS[i]: int(r[i]) for i in range(6)}

    def decode(self, gid):
        e = Expr()
        _check(lib().dse_decode(self._h, gid, C.byref(e)))
        return e.rung, e.op, e.a, e.b

    def expr(self, gid) -> str:
        buf = C.create_string_buffer(1 << 14)
        _check(lib().dse_expr_string(self._h, gid, buf, len(buf)))
        return buf.value.decode()

    def candidate_units(self, ids):
        """(units int64 [n, n_dims] scaled by 2^max_rung, unit_ok int8 [n]) of
        the candidate ids (dse_candidate_units)."""
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        n = len(ids)
        units = np.zeros((n, max(self.n_dims, 1)), np.int64)
        ok = np.zeros(n, np.int8)
        _check(lib().dse_candidate_units(self._h, ids.ctypes.data, n, units.ctypes.data, ok.ctypes.data))
        return units[:, : self.n_dims], ok

    def screen(self, Y, k, mode=MODE_PER_TARGET, precision=PREC_FP32, id_begin=0, id_end=0, stream=None,
               flags=0, dedup_tau=None, reasons=None, intervals=None) -> Result:
        """SIS screen (dse_sis_screen).  With ``dedup_tau`` (0 < tau < 0.5) the
        lists hold the top-k of the non-redundant candidates (DSE_FLAG_DEDUP).
        ``reasons``: optional torch int8 CUDA tensor of id_end - id_begin
        entries that receives the reason code of every screened candidate.
        ``intervals``: optional torch float32 CUDA tensor of
        (id_end - id_begin) x n_lists x 2 entries that receives each
        candidate's pre-re-score (score, bound) per list (NaN where none)."""
        if dedup_tau is not None:
            flags |= FLAG_DEDUP
        if isinstance(Y, np.ndarray):
            Y = np.ascontiguousarray(np.atleast_2d(Y), dtype=np.float64)
        elif Y.dim() == 1:
            Y = Y.reshape(1, -1)
        T, ldy = Y.shape
        py, ydev = _ptr(Y)
        self._ykeep = Y
        pw = None
        if reasons is not None:
            pw, wdev = _ptr(reasons)
            if not wdev:
                raise ValueError("reasons must be a CUDA tensor")
        pv = None
        if intervals is not None:
            pv, vdev = _ptr(intervals)
            if not vdev:
                raise ValueError("intervals must be a CUDA tensor")
        d = ScreenDesc(py, ldy, ydev, T, k, mode, precision, id_begin, id_end, stream, flags, 0,
                       dedup_tau if dedup_tau is not None else 0.0, pw, pv)
        h = C.c_void_p()
        _check(lib().dse_sis_screen(self._h, C.byref(d), C.byref(h)))
        return Result(h, 1 if mode == MODE_AGGREGATED else T, k)

    def residual_loop(self, y, n_iter, k, precision=PREC_FP32, sis_ids=None, residual=None, stream=None, flags=0,
                      fixed=()):
        """The residual loop on the device (dse_residual_loop): returns a dict
        with the chosen ids, RMSEs, coefficients and per-iteration screen
        statistics.  ``sis_ids`` / ``residual``: optional output buffers
        (numpy or torch CUDA) of n_iter*k ids and N values.  ``fixed``:
        descriptors already chosen (resume after len(fixed) iterations)."""
        if isinstance(y, np.ndarray):
            y = np.ascontiguousarray(y, dtype=np.float64)
        py, ydev = _ptr(y)
        fx = np.ascontiguousarray(np.asarray(fixed, dtype=np.uint64))
        d = LoopDesc(py, ydev, n_iter, k, precision, flags, stream, len(fx), 0, fx.ctypes.data if len(fx) else None)
        out = LoopResult()
        pi, _ = _ptr(sis_ids)
        pr, _ = _ptr(residual)
        _check(lib().dse_residual_loop(self._h, C.byref(d), C.byref(out), pi, pr))
        return {"chosen": [int(out.chosen[i]) for i in range(n_iter)],
                "rmse": [float(out.rmse[i]) for i in range(n_iter)],
                "coefs": [[float(out.coefs[i][c]) for c in range(i + 2)] for i in range(n_iter)],
                "stats": [_stats_dict(out.stats[i]) for i in range(n_iter)]}

    def l0_search(self, y, ids, dim, n_top=16, stream=None):
        """Exhaustive L0 search over the listed candidates (dse_l0_search):
        (positions int64[m, dim], RMSE[m], coefficients[m, dim+1]) of the m
        best subsets by (RMSE, positions)."""
        if isinstance(y, np.ndarray):
            y = np.ascontiguousarray(y, dtype=np.float64)
        if isinstance(ids, np.ndarray):
            ids = np.ascontiguousarray(ids, dtype=np.uint64)
        py, ydev = _ptr(y)
        pi, idev = _ptr(ids)
        n = len(ids) if isinstance(ids, np.ndarray) else ids.numel()
        d = L0Desc(py, ydev, dim, pi, n, idev, n_top, stream)
        pos = np.zeros((n_top, dim), np.int64)
        rm = np.zeros(n_top)
        cf = np.zeros((n_top, dim + 1))
        nf = C.c_int32()
        _check(lib().dse_l0_search(self._h, C.byref(d), pos.ctypes.data, rm.ctypes.data, cf.ctypes.data,
                                   C.byref(nf)))
        m = nf.value
        return pos[:m].copy(), rm[:m].copy(), cf[:m].copy()

    def ls_refit(self, y, fixed, cand, residual=None, stream=None):
        """Best candidate for the next descriptor slot: (id, rmse, coefs, residual)."""
        if isinstance(y, np.ndarray):
            y = np.ascontiguousarray(y, dtype=np.float64)
        fixed = np.ascontiguousarray(fixed, dtype=np.uint64)
        if isinstance(cand, np.ndarray):
            cand = np.ascontiguousarray(cand, dtype=np.uint64)
        py, ydev = _ptr(y)
        pc, cdev = _ptr(cand)
        ncand = len(cand) if isinstance(cand, np.ndarray) else cand.numel()
        d = RefitDesc(py, ydev, len(fixed), fixed.ctypes.data if len(fixed) else None, pc, ncand, cdev, 0, stream)
        bid, brm = C.c_uint64(), C.c_double()
        coefs = np.zeros(len(fixed) + 2)
        if residual is None:
            residual = np.zeros(self.n_samples)
        pr, _ = _ptr(residual)
        _check(lib().dse_ls_refit(self._h, C.byref(d), C.byref(bid), C.byref(brm), coefs.ctypes.data, pr))
        return int(bid.value), float(brm.value), coefs, residual

    def ls_refit_noalloc(self, y, fixed, cand, residual=None, stream=None):
        """Same as ls_refit through dse_ls_refit_noalloc, which allocates no
        device memory: for callers that cannot allocate while they run (an
        external memory pool or a hard budget owns the device).  It waits for
        the stream like ls_refit, so it is not for a capturing stream.  Fixed
        limits: N <= 32768 samples, at most 16384 candidates; one shared
        scratch area per device, so overlapping calls must be serialised by
        the caller."""
        if isinstance(y, np.ndarray):
            y = np.ascontiguousarray(y, dtype=np.float64)
        fixed = np.ascontiguousarray(fixed, dtype=np.uint64)
        if isinstance(cand, np.ndarray):
            cand = np.ascontiguousarray(cand, dtype=np.uint64)
        py, ydev = _ptr(y)
        pc, cdev = _ptr(cand)
        ncand = len(cand) if isinstance(cand, np.ndarray) else cand.numel()
        d = RefitDesc(py, ydev, len(fixed), fixed.ctypes.data if len(fixed) else None, pc, ncand, cdev, 0, stream)
        bid, brm = C.c_uint64(), C.c_double()
        coefs = np.zeros(len(fixed) + 2)
        if residual is None:
            residual = np.zeros(self.n_samples)
        pr, _ = _ptr(residual)
        _check(lib().dse_ls_refit_noalloc(self._h, C.byref(d), C.byref(bid), C.byref(brm), coefs.ctypes.data, pr))
        return int(bid.value), float(brm.value), coefs, residual
