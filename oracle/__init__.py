"""CPU oracle for the hash-based multi-phase SpGEMM (arXiv 2512.12036).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers. The library path never imports this
package, and this package imports nothing from the library; the two share
only the seeded input generators.

The SpGEMM arithmetic lives in ``oracle.c`` (plain C, fp64, optional OpenMP
over rows); this module builds it with gcc on first use and marshals numpy
arrays. Which passage of the paper each function restates is given in
``oracle.c``. The pruned GNN layer (``layers.py``) and bulk sampling
(``sampling.py``) are plain numpy in fp64 on small inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ORACLE_C_SOURCE names another copy of oracle.c, built next to that copy:
# the mutation test uses it to check that the pins catch planted mistakes
_SRC = os.environ.get("ORACLE_C_SOURCE") or os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(_SRC)), "liboracle.so")
_lock = threading.Lock()
_lib = None

i32p = ctypes.POINTER(ctypes.c_int32)
i64p = ctypes.POINTER(ctypes.c_int64)
f32p = ctypes.POINTER(ctypes.c_float)
f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.orc_ip_count.restype = ctypes.c_int64
            L.orc_ip_count.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i64p]
            L.orc_group_rows.restype = None
            L.orc_group_rows.argtypes = [ctypes.c_int32, i64p, ctypes.c_int32, i64p, i32p, i32p]
            L.orc_symbolic.restype = ctypes.c_int
            L.orc_symbolic.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p, i32p,
                                       i32p, ctypes.c_int32, i32p, ctypes.c_int]
            L.orc_numeric.restype = ctypes.c_int
            L.orc_numeric.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, f32p, i32p, i32p,
                                      f32p, i32p, ctypes.c_int32, i64p, i32p, f64p, f64p, ctypes.c_int]
            L.orc_backward.restype = ctypes.c_int
            L.orc_backward.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, f32p,
                                       ctypes.c_int32, i32p, i32p, f32p, i64p, i32p, f64p, f64p, f64p]
            L.orc_mcl_step.restype = ctypes.c_int64
            L.orc_mcl_step.argtypes = [ctypes.c_int32, i64p, i32p, f32p, ctypes.c_double,
                                       ctypes.c_int32, ctypes.c_double, ctypes.c_int32, i64p, i32p, f64p]
            L.orc_row_normalise.restype = None
            L.orc_row_normalise.argtypes = [ctypes.c_int32, i64p, f32p, f64p]
            L.orc_max_threads.restype = ctypes.c_int
            L.orc_max_threads.argtypes = []
            _lib = L
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def max_threads() -> int:
    return int(lib().orc_max_threads())


@dataclass
class OracleCSR:
    """Oracle output: int64 row pointers, int32 sorted columns, fp64 values and
    the per-entry error scale sum |a||b| (``bound``)."""

    rows: int
    cols: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    bound: np.ndarray | None = None

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])


def ip_count(A, B):
    """Algorithm 1: (IP per row as int64, total)."""
    rptA, colA, rptB = _c(A.row_ptr, np.int32), _c(A.col, np.int32), _c(B.row_ptr, np.int32)
    ip = np.zeros(A.rows, dtype=np.int64)
    total = lib().orc_ip_count(A.rows, _p(rptA, i32p), _p(colA, i32p), _p(rptB, i32p), _p(ip, i64p))
    return ip, int(total)


def group_rows(key: np.ndarray, thresholds):
    """Section III-B grouping: (map, offsets) with groups split at ``thresholds``."""
    key = _c(key, np.int64)
    thr = _c(np.asarray(thresholds, dtype=np.int64), np.int64)
    m = key.shape[0]
    mp = np.zeros(m, dtype=np.int32)
    off = np.zeros(thr.shape[0] + 2, dtype=np.int32)
    lib().orc_group_rows(m, _p(key, i64p), thr.shape[0], _p(thr, i64p), _p(mp, i32p), _p(off, i32p))
    return mp, off


def symbolic(A, B, rows=None, nthreads: int = 0) -> np.ndarray:
    """nnz of each output row (of ``rows`` when given)."""
    rptA, colA = _c(A.row_ptr, np.int32), _c(A.col, np.int32)
    rptB, colB = _c(B.row_ptr, np.int32), _c(B.col, np.int32)
    rl = None if rows is None else _c(rows, np.int32)
    n = A.rows if rl is None else rl.shape[0]
    out = np.zeros(n, dtype=np.int32)
    rc = lib().orc_symbolic(A.rows, B.cols, _p(rptA, i32p), _p(colA, i32p), _p(rptB, i32p),
                            _p(colB, i32p), _p(rl, i32p), n, _p(out, i32p), nthreads)
    if rc != 0:
        raise ValueError("oracle: column index out of range")
    return out


def spgemm(A, B, rows=None, nthreads: int = 0, with_bound: bool = True) -> OracleCSR:
    """C = A*B (or the listed rows of it) in fp64, sorted columns, plus bounds."""
    nnz = symbolic(A, B, rows, nthreads)
    ptr = np.zeros(nnz.shape[0] + 1, dtype=np.int64)
    np.cumsum(nnz, out=ptr[1:])
    total = int(ptr[-1])
    col = np.zeros(total, dtype=np.int32)
    val = np.zeros(total, dtype=np.float64)
    bnd = np.zeros(total, dtype=np.float64) if with_bound else None
    rptA, colA, valA = _c(A.row_ptr, np.int32), _c(A.col, np.int32), _c(A.val, np.float32)
    rptB, colB, valB = _c(B.row_ptr, np.int32), _c(B.col, np.int32), _c(B.val, np.float32)
    rl = None if rows is None else _c(rows, np.int32)
    n = nnz.shape[0]
    rc = lib().orc_numeric(A.rows, B.cols, _p(rptA, i32p), _p(colA, i32p), _p(valA, f32p),
                           _p(rptB, i32p), _p(colB, i32p), _p(valB, f32p), _p(rl, i32p), n,
                           _p(ptr, i64p), _p(col, i32p), _p(val, f64p), _p(bnd, f64p), nthreads)
    if rc != 0:
        raise ValueError("oracle: inconsistent input")
    return OracleCSR(n, B.cols, ptr, col, val, bnd)


def backward(A, B, C: OracleCSR, dC: np.ndarray, want_dA: bool = True, want_dB: bool = True):
    """Gradients of sum(dC * C) with respect to A's and B's stored values (fp64)."""
    rptA, colA, valA = _c(A.row_ptr, np.int32), _c(A.col, np.int32), _c(A.val, np.float32)
    rptB, colB, valB = _c(B.row_ptr, np.int32), _c(B.col, np.int32), _c(B.val, np.float32)
    rptC, colC, g = _c(C.row_ptr, np.int64), _c(C.col, np.int32), _c(dC, np.float64)
    dA = np.zeros(A.nnz, dtype=np.float64) if want_dA else None
    dB = np.zeros(B.nnz, dtype=np.float64) if want_dB else None
    rc = lib().orc_backward(A.rows, B.cols, _p(rptA, i32p), _p(colA, i32p), _p(valA, f32p),
                            B.rows, _p(rptB, i32p), _p(colB, i32p), _p(valB, f32p),
                            _p(rptC, i64p), _p(colC, i32p), _p(g, f64p), _p(dA, f64p), _p(dB, f64p))
    if rc != 0:
        raise ValueError("oracle: C structure does not cover the product")
    return dA, dB


def mcl_step(M, theta: float, k: int, r: float, order: int = 0) -> OracleCSR:
    """Prune / top-k / inflate / normalise on the rows of M^T (Algorithm 6)."""
    rpt = _c(M.row_ptr, np.int64)
    col = _c(M.col, np.int32)
    val = _c(M.val, np.float32)
    nnz = col.shape[0]
    optr = np.zeros(M.rows + 1, dtype=np.int64)
    ocol = np.zeros(max(nnz, 1), dtype=np.int32)
    oval = np.zeros(max(nnz, 1), dtype=np.float64)
    n = lib().orc_mcl_step(M.rows, _p(rpt, i64p), _p(col, i32p), _p(val, f32p), theta, k, r,
                           order, _p(optr, i64p), _p(ocol, i32p), _p(oval, f64p))
    return OracleCSR(M.rows, M.cols, optr, ocol[:n].copy(), oval[:n].copy())


def row_normalise(M) -> np.ndarray:
    """Each stored value over its row sum, fp64 (column normalisation of M held as M^T)."""
    rpt = _c(M.row_ptr, np.int64)
    val = _c(M.val, np.float32)
    out = np.zeros(val.shape[0], dtype=np.float64)
    lib().orc_row_normalise(M.rows, _p(rpt, i64p), _p(val, f32p), _p(out, f64p))
    return out
