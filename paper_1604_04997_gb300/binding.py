"""Thin ctypes binding of the C ABI in ``include/pm.h`` (argument marshalling only).

Device buffers are passed as raw pointers (``tensor.data_ptr()``); streams as
``torch.cuda.Stream.cuda_stream`` integers.  Every computation happens in the
library's CUDA kernels; if the library is missing this module raises instead of
computing anything itself.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpm.so")

PM_OK = 0
PM_PENDING = 2
PM_WARN_RANK_DEFICIENT = 1
ERRORS = {-1: "PM_ERR_INVALID_ARG", -2: "PM_ERR_PARSE", -3: "PM_ERR_UNSUPPORTED", -4: "PM_ERR_OVERFLOW_RANGE",
          -5: "PM_ERR_NOMEM", -6: "PM_ERR_BUSY", -7: "PM_ERR_TIMEOUT", -8: "PM_ERR_CUDA",
          -9: "PM_ERR_OUT_OF_BOX", -10: "PM_ERR_NOT_FOUND"}
PREC_FP64, PREC_BF16X3, PREC_NATIVE_FP64 = 0, 1, 2
FIT_RELATIVE, FIT_ABSOLUTE = 0, 1

_lib = None


class PMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class TableInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("n_params", "n_atoms", "n_conds", "n_pieces", "n_monomials", "n_columns", "n_words", "degree")]


class FitReport(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("n_dropped", ctypes.c_int32), ("cond_est", ctypes.c_double), ("rel_resid", ctypes.c_double),
                ("last_update", ctypes.c_double)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("batch_interval_us", ctypes.c_int32), ("n_streams", ctypes.c_int32),
                ("max_batch_queries", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Query(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("topk", ctypes.c_int32), ("n_cand", ctypes.c_int64),
                ("h_tables", ctypes.c_void_p), ("h_points", ctypes.c_void_p),
                ("h_top_idx", ctypes.c_void_p), ("h_top_t", ctypes.c_void_p)]


class PmmConfig(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("variant", ctypes.c_int32), ("k", ctypes.c_int32), ("gx", ctypes.c_int32),
                ("gy", ctypes.c_int32), ("f64", ctypes.c_int32), ("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("l", ctypes.c_int64)]


PMM_KINDS = ("empty", "copy", "sum4", "index", "vsa", "filled", "arith", "transpose_p", "transpose_r", "transpose_w",
             "matmul", "matmul_naive", "stencil", "matvec", "reduction", "axpy", "vecadd", "nbody", "conv5")


class ServeStats(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_int64), ("n_batches", ctypes.c_int64), ("n_candidates", ctypes.c_int64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("max_us", ctypes.c_double),
                ("mean_us", ctypes.c_double), ("n_rejected", ctypes.c_int64), ("h2d_bytes", ctypes.c_int64),
                ("d2h_bytes", ctypes.c_int64)]


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        sig = {
            "pm_create": ([ctypes.POINTER(vp), ctypes.c_int, sz], i32),
            "pm_destroy": ([vp], None),
            "pm_last_error": ([], ctypes.c_char_p),
            "pm_sync_status": ([vp, vp], i32),
            "pm_compile_counts": ([vp, ctypes.c_char_p, sz, i32, vp, vp, ctypes.POINTER(i32),
                                   ctypes.POINTER(TableInfo)], i32),
            "pm_table_image": ([vp, i32, vp, sz, ctypes.POINTER(sz)], i32),
            "pm_eval_counts": ([vp, vp, i32, vp, i64, vp, vp], i32),
            "pm_predict": ([vp, vp, i64, i32, vp, i32, i32, vp, vp], i32),
            "pm_predict_argmin": ([vp, vp, i64, i32, vp, i32, i32, vp, vp, vp], i32),
            "pm_predict_argmin_static": ([vp, i64, i32, vp, i32, vp, vp, vp], i32),
            "pm_eval_predict_topk": ([vp, vp, vp, i32, vp, vp, vp, i32, vp, vp, vp], i32),
            "pm_tune": ([vp, i32, ctypes.c_char_p], i32),
            "pm_plan_info": ([vp, vp, vp, i32, vp, vp], i32),
            "pm_plan_tune_log": ([vp, vp, vp, i32, vp, vp, i32], i32),
            "pm_fit_weights": ([vp, vp, i64, i32, vp, i32, i32, i32, i32, vp, ctypes.POINTER(FitReport), vp], i32),
            "pm_serve_set_weights": ([vp, vp, i32], i32),
            "pm_serve_start": ([vp, ctypes.POINTER(ServeConfig)], i32),
            "pm_serve_submit": ([vp, ctypes.POINTER(Query), ctypes.POINTER(ctypes.c_uint64)], i32),
            "pm_serve_poll": ([vp, ctypes.c_uint64, i32], i32),
            "pm_serve_stats": ([vp, i32, ctypes.POINTER(ServeStats)], i32),
            "pm_serve_stop": ([vp], i32),
            "pmm_time": ([ctypes.POINTER(PmmConfig), i32, i32, ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_double), vp], i32),
            "pmm_int_issue_rate": ([ctypes.POINTER(ctypes.c_double), vp], i32),
            "pm_table_load": ([vp, vp, ctypes.c_size_t, ctypes.POINTER(i32)], i32),
            "pm_predict_topk": ([vp, vp, ctypes.c_int64, i32, vp, i32, i32, vp, i32, vp, i32, vp, vp, vp], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols() -> Sequence[str]:
    return ("pm_create", "pm_destroy", "pm_last_error", "pm_sync_status", "pm_compile_counts", "pm_table_image",
            "pm_eval_counts", "pm_predict", "pm_predict_argmin", "pm_predict_argmin_static",
            "pm_eval_predict_topk", "pm_tune",
            "pm_plan_info", "pm_plan_tune_log", "pm_fit_weights", "pm_serve_set_weights", "pm_serve_start", "pm_serve_submit",
            "pm_serve_poll", "pm_serve_stats", "pm_serve_stop", "pmm_time", "pmm_int_issue_rate", "pm_table_load",
            "pm_predict_topk")


def _check(rc: int, ok=(PM_OK,)) -> int:
    if rc in ok:
        return rc
    raise PMError(rc, lib().pm_last_error().decode())


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover
            return None
    return stream if isinstance(stream, int) else stream.cuda_stream


class Context:
    """A pm_ctx.  device = -1 gives a host-only context (compilation only)."""

    def __init__(self, device: int = 0, mem_budget: int = 0):
        h = ctypes.c_void_p()
        _check(lib().pm_create(ctypes.byref(h), device, mem_budget))
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            lib().pm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- counting
    def compile_counts(self, ir: str, layout: int, lo: Sequence[int], hi: Sequence[int]) -> Tuple[int, dict]:
        b = ir.encode()
        lo_a = np.ascontiguousarray(lo, dtype=np.int64)
        hi_a = np.ascontiguousarray(hi, dtype=np.int64)
        tid = ctypes.c_int32()
        info = TableInfo()
        _check(lib().pm_compile_counts(self.h, b, len(b), layout, lo_a.ctypes.data, hi_a.ctypes.data,
                                       ctypes.byref(tid), ctypes.byref(info)))
        return tid.value, {f: getattr(info, f) for f, _ in TableInfo._fields_}

    def table_load(self, words) -> int:
        """Register a table from its image (as table_image returns it); the image is
        checked on the host and refused with PMError if it is not a valid table."""
        w = np.ascontiguousarray(words, dtype=np.uint32)
        tid = ctypes.c_int32()
        _check(lib().pm_table_load(self.h, w.ctypes.data, w.size, ctypes.byref(tid)))
        return tid.value

    def table_image(self, tid: int) -> np.ndarray:
        n = ctypes.c_size_t()
        _check(lib().pm_table_image(self.h, tid, None, 0, ctypes.byref(n)))
        buf = np.zeros(n.value, dtype=np.uint32)
        _check(lib().pm_table_image(self.h, tid, buf.ctypes.data, n.value, ctypes.byref(n)))
        return buf

    def eval_counts(self, ids: Sequence[int], points, out, stream=None):
        ids_a = np.ascontiguousarray(ids, dtype=np.int32)
        _check(lib().pm_eval_counts(self.h, ids_a.ctypes.data, len(ids_a), _ptr(points), points.shape[0],
                                    _ptr(out), _stream(stream)))

    def sync_status(self, stream=None):
        _check(lib().pm_sync_status(self.h, _stream(stream)))

    # -- prediction
    def predict(self, F, W, T, precision: int = PREC_FP64, stream=None):
        _check(lib().pm_predict(self.h, _ptr(F), F.shape[0], F.shape[1], _ptr(W), W.shape[0], precision, _ptr(T),
                                _stream(stream)))

    def predict_argmin(self, F, W, arg, mn, precision: int = PREC_FP64, stream=None):
        _check(lib().pm_predict_argmin(self.h, _ptr(F), F.shape[0], F.shape[1], _ptr(W), W.shape[0], precision,
                                       _ptr(arg), _ptr(mn), _stream(stream)))

    def predict_topk(self, F, W, seg_off, topk, top_idx, top_t, rows=None, precision: int = PREC_FP64, stream=None):
        """Top-k rows per (group, model); seg_off: host int64 [G+1] group offsets into
        rows (device int64 row list) or, with rows None, into F's rows."""
        so = np.ascontiguousarray(seg_off, dtype=np.int64)
        _check(lib().pm_predict_topk(self.h, _ptr(F), F.shape[0], F.shape[1], _ptr(W), W.shape[0], precision,
                                     so.ctypes.data, so.size - 1, _ptr(rows), topk, _ptr(top_idx), _ptr(top_t),
                                     _stream(stream)))

    def eval_predict_topk(self, tables, var_off, points, pt_off, w, topk, top_idx, top_t, stream=None):
        t = np.ascontiguousarray(tables, dtype=np.int32)
        vo = np.ascontiguousarray(var_off, dtype=np.int32)
        po = np.ascontiguousarray(pt_off, dtype=np.int64)
        _check(lib().pm_eval_predict_topk(self.h, t.ctypes.data, vo.ctypes.data, len(vo) - 1, _ptr(points),
                                          po.ctypes.data, _ptr(w), topk, _ptr(top_idx), _ptr(top_t),
                                          _stream(stream)))

    def tune(self, enable: bool, cache_path: Optional[str] = None):
        _check(lib().pm_tune(self.h, int(enable), cache_path.encode() if cache_path else None))

    def plan_info(self, tables, var_off, pt_off) -> dict:
        t = np.ascontiguousarray(tables, dtype=np.int32)
        vo = np.ascontiguousarray(var_off, dtype=np.int32)
        po = np.ascontiguousarray(pt_off, dtype=np.int64)
        out = np.zeros(8, dtype=np.int64)
        _check(lib().pm_plan_info(self.h, t.ctypes.data, vo.ctypes.data, len(vo) - 1, po.ctypes.data,
                                  out.ctypes.data))
        return dict(units=int(out[0]), evals=int(out[1]), work_per_eval=out[2] / 1000.0, nw=int(out[3]),
                    grid=int(out[4]), tuned=bool(out[5]), groups=int(out[6]), slice=int(out[7]))

    def plan_tune_log(self, tables, var_off, pt_off) -> list:
        """The autotuner's candidates: (slice, warps per CTA, CTAs per SM, ms)."""
        t = np.ascontiguousarray(tables, dtype=np.int32)
        vo = np.ascontiguousarray(var_off, dtype=np.int32)
        po = np.ascontiguousarray(pt_off, dtype=np.int64)
        out = np.zeros((64, 4), dtype=np.float64)
        n = lib().pm_plan_tune_log(self.h, t.ctypes.data, vo.ctypes.data, len(vo) - 1, po.ctypes.data,
                                   out.ctypes.data, 64)
        return [tuple(r) for r in out[:max(0, min(n, 64))]]

    # -- fit
    def fit_weights(self, F, T, W_out, objective=FIT_RELATIVE, precision=PREC_BF16X3, refine_steps=3, stream=None):
        M = T.shape[1]
        rep = (FitReport * M)()
        rc = _check(lib().pm_fit_weights(self.h, _ptr(F), F.shape[0], F.shape[1], _ptr(T), M, objective, precision,
                                         refine_steps, _ptr(W_out), rep, _stream(stream)),
                    ok=(PM_OK, PM_WARN_RANK_DEFICIENT))
        return rc, [{f: getattr(r, f) for f, _ in FitReport._fields_} for r in rep]

    # -- serving
    def serve_set_weights(self, W: np.ndarray):
        W = np.ascontiguousarray(W, dtype=np.float64)
        _check(lib().pm_serve_set_weights(self.h, W.ctypes.data, W.shape[0]))

    def serve_start(self, batch_interval_us=200, n_streams=2, max_batch_queries=256):
        cfg = ServeConfig(batch_interval_us, n_streams, max_batch_queries, 0)
        _check(lib().pm_serve_start(self.h, ctypes.byref(cfg)))

    def serve_submit(self, q: Query) -> int:
        t = ctypes.c_uint64()
        _check(lib().pm_serve_submit(self.h, ctypes.byref(q), ctypes.byref(t)))
        return t.value

    def serve_poll(self, ticket: int, timeout_us: int = 0) -> int:
        return _check(lib().pm_serve_poll(self.h, ticket, timeout_us), ok=(PM_OK, PM_PENDING))

    def serve_stats(self, reset: bool = False) -> dict:
        st = ServeStats()
        _check(lib().pm_serve_stats(self.h, int(reset), ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServeStats._fields_}

    def serve_stop(self):
        _check(lib().pm_serve_stop(self.h))


def pmm_time(kind: str, variant: int = 0, k: int = 0, gx: int = 256, gy: int = 1, n: int = 1, m: int = 0,
             l: int = 0, runs: int = 30, skip: int = 4, stream=None, f64: bool = False) -> Tuple[float, float]:
    """Time one measurement-kernel configuration (include/pm_measure.h): (min, mean) ms
    over runs - skip timed runs."""
    cfg = PmmConfig(PMM_KINDS.index(kind), variant, k, gx, gy, int(f64), n, m, l)
    mn, me = ctypes.c_double(), ctypes.c_double()
    _check(lib().pmm_time(ctypes.byref(cfg), runs, skip, ctypes.byref(mn), ctypes.byref(me), _stream(stream)))
    return mn.value, me.value


def pmm_int_issue_rate(stream=None) -> float:
    """Measured integer issue rate of the current GPU (lane operations per second)."""
    v = ctypes.c_double()
    _check(lib().pmm_int_issue_rate(ctypes.byref(v), _stream(stream)))
    return v.value


def make_query(model: int, topk: int, tables: np.ndarray, points: np.ndarray, top_idx: np.ndarray,
               top_t: np.ndarray) -> Query:
    """A pm_query over host arrays; the caller keeps the arrays alive until the poll."""
    assert tables.dtype == np.int32 and points.dtype == np.int64 and points.shape[1:] == (4,)
    assert top_idx.dtype == np.int32 and top_t.dtype == np.float64 and len(top_idx) >= topk
    return Query(model, topk, len(tables), tables.ctypes.data if len(tables) else None,
                 points.ctypes.data if len(tables) else None, top_idx.ctypes.data, top_t.ctypes.data)


def predict_argmin_static(F, W, arg, mn, stream=None):
    """pm_predict_argmin_static: needs no context and allocates no device memory."""
    _check(lib().pm_predict_argmin_static(_ptr(F), F.shape[0], F.shape[1], _ptr(W), W.shape[0], _ptr(arg),
                                          _ptr(mn), _stream(stream)))
