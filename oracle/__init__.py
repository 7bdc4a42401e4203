"""Python access to the C oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by
the CPU-baseline leg of ``bench.py``.  The library in ``paper_1604_04997_gb300`` never
imports it, and the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

NKEYS = 17 + 2 * 3 * 15
CLASS_NAMES = ["0", "1", "1/2", "2/2", "1/3", "2/3", "3/3", "1/4", "2/4", "3/4", "4/4",
               "1/>4", "2/>4", "3/>4", "4/>4"]


def build(force: bool = False) -> str:
    """Compile the oracle for this machine (plain gcc, OpenMP, no fp contraction so
    the error-free transformations stay exact)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src),
                                                   os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-Wno-unused-function", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P, I64P, I32P, DP = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), \
                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)
            L.orc_parse.restype = P
            L.orc_parse.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int]
            L.orc_free.argtypes = [P]
            L.orc_n_params.argtypes = [P]
            L.orc_n_stmts.argtypes = [P]
            L.orc_n_access.argtypes = [P, ctypes.c_int]
            L.orc_classify.argtypes = [P, I32P, ctypes.c_int]
            L.orc_count_brute.argtypes = [P, I64P, ctypes.c_int64, I64P]
            L.orc_count_struct.argtypes = [P, I64P, I64P]
            L.orc_layout.argtypes = [I64P, ctypes.c_int, I64P]
            L.orc_eval.argtypes = [P, ctypes.c_int, ctypes.c_int, I64P, ctypes.c_int64, ctypes.c_int64, I64P]
            L.orc_predict.argtypes = [I64P, ctypes.c_int64, ctypes.c_int, DP, ctypes.c_int, DP]
            L.orc_predict_abs.argtypes = [I64P, ctypes.c_int64, ctypes.c_int, DP, ctypes.c_int, DP]
            L.orc_topk.argtypes = [DP, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, I32P, DP]
            L.orc_fit.argtypes = [I64P, ctypes.c_int64, ctypes.c_int, DP, ctypes.c_int, DP, DP]
            L.orc_eval_predict_topk.argtypes = [ctypes.POINTER(P), ctypes.c_int, I64P, ctypes.c_int64,
                                                DP, ctypes.c_int, I32P, DP, ctypes.c_int]
            _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class OracleError(RuntimeError):
    pass


class Kernel:
    """A parsed IR kernel held by the oracle."""

    def __init__(self, text: str):
        L = lib()
        err = ctypes.create_string_buffer(256)
        self._h = L.orc_parse(text.encode(), err, 256)
        if not self._h:
            raise OracleError(err.value.decode())
        self.n_params = L.orc_n_params(self._h)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_free(self._h)
            self._h = None

    def classes(self) -> List[List[int]]:
        L = lib()
        buf = np.zeros(4096, dtype=np.int32)
        n = L.orc_classify(self._h, _p(buf, ctypes.c_int32), len(buf))
        if n < 0:
            raise OracleError(f"classification failed ({n})")
        out, q = [], 0
        for s in range(L.orc_n_stmts(self._h)):
            na = L.orc_n_access(self._h, s)
            out.append([int(x) for x in buf[q:q + na]])
            q += na
        return out

    def keys(self, params: Sequence[int], method: str = "brute", max_points: int = 1 << 26) -> np.ndarray:
        L = lib()
        par = np.ascontiguousarray(params, dtype=np.int64)
        out = np.zeros(NKEYS, dtype=np.int64)
        if method == "brute":
            r = L.orc_count_brute(self._h, _p(par, ctypes.c_int64), max_points, _p(out, ctypes.c_int64))
        else:
            r = L.orc_count_struct(self._h, _p(par, ctypes.c_int64), _p(out, ctypes.c_int64))
        if r:
            raise OracleError(f"count failed ({r})")
        return out

    def features(self, points: np.ndarray, layout: int = 32, method: str = "struct",
                 max_points: int = 1 << 26) -> np.ndarray:
        L = lib()
        pts = np.ascontiguousarray(points, dtype=np.int64).reshape(-1, self.n_params)
        out = np.zeros((len(pts), layout), dtype=np.int64)
        r = L.orc_eval(self._h, layout, 0 if method == "brute" else 1, _p(pts, ctypes.c_int64),
                       len(pts), max_points, _p(out, ctypes.c_int64))
        if r:
            raise OracleError(f"eval failed ({r})")
        return out


def layout(keys: np.ndarray, k: int) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    out = np.zeros(k, dtype=np.int64)
    if lib().orc_layout(_p(keys, ctypes.c_int64), k, _p(out, ctypes.c_int64)) != k:
        raise OracleError("bad layout")
    return out


def predict(F: np.ndarray, W: np.ndarray) -> np.ndarray:
    F = np.ascontiguousarray(F, dtype=np.int64)
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    R, k = F.shape
    M = W.shape[0]
    T = np.zeros((R, M), dtype=np.float64)
    lib().orc_predict(_p(F, ctypes.c_int64), R, k, _p(W, ctypes.c_double), M, _p(T, ctypes.c_double))
    return T


def predict_abs(F: np.ndarray, W: np.ndarray) -> np.ndarray:
    F = np.ascontiguousarray(F, dtype=np.int64)
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    R, k = F.shape
    M = W.shape[0]
    A = np.zeros((R, M), dtype=np.float64)
    lib().orc_predict_abs(_p(F, ctypes.c_int64), R, k, _p(W, ctypes.c_double), M, _p(A, ctypes.c_double))
    return A


def topk(t: np.ndarray, k: int):
    """t [groups][seg] -> (idx [groups][k], val [groups][k]) ordered by (t, index)."""
    t = np.ascontiguousarray(np.atleast_2d(t), dtype=np.float64)
    G, S = t.shape
    idx = np.zeros((G, k), dtype=np.int32)
    val = np.zeros((G, k), dtype=np.float64)
    lib().orc_topk(_p(t, ctypes.c_double), G, S, k, _p(idx, ctypes.c_int32), _p(val, ctypes.c_double))
    return idx, val


def fit(F: np.ndarray, t: np.ndarray, objective: str = "relative"):
    """Fit one weight vector; returns (w[k], rank, cond_estimate, rel_residual)."""
    F = np.ascontiguousarray(F, dtype=np.int64)
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
    R, k = F.shape
    w = np.zeros(k, dtype=np.float64)
    rep = np.zeros(3, dtype=np.float64)
    r = lib().orc_fit(_p(F, ctypes.c_int64), R, k, _p(t, ctypes.c_double),
                      0 if objective == "relative" else 1, _p(w, ctypes.c_double), _p(rep, ctypes.c_double))
    if r < 0:
        raise OracleError("fit failed")
    return w, int(rep[0]), float(rep[1]), float(rep[2])


def eval_predict_topk(kernels: Sequence[Kernel], points: np.ndarray, w: np.ndarray, topk_: int,
                      n_threads: int = 0):
    """CPU baseline of the batched tuning workload for one template."""
    pts = np.ascontiguousarray(points, dtype=np.int64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    H = (ctypes.c_void_p * len(kernels))(*[k._h for k in kernels])
    n = len(pts)
    idx = np.zeros((n, topk_), dtype=np.int32)
    val = np.zeros((n, topk_), dtype=np.float64)
    r = lib().orc_eval_predict_topk(H, len(kernels), _p(pts, ctypes.c_int64), n, _p(w, ctypes.c_double),
                                    topk_, _p(idx, ctypes.c_int32), _p(val, ctypes.c_double), n_threads)
    if r:
        raise OracleError(f"eval_predict_topk failed ({r})")
    return idx, val
