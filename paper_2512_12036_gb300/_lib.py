"""ctypes loader for libspgemm.so: the C ABI declared in include/spgemm.h.

There is no fallback: if the shared library cannot be built or loaded, the
import fails with the reason.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_vp = ctypes.c_void_p
c_sz = ctypes.c_size_t

OK = 0
ERR_INVALID = 1
ERR_WORKSPACE = 2
ERR_OVERFLOW = 3
ERR_BUDGET = 4
ERR_TIMEOUT = 5
ERR_CUDA = 6
ERR_INTERNAL = 7
ERR_UNSUPPORTED = 8


class CsrStruct(ctypes.Structure):
    _fields_ = [("rows", c_i32), ("cols", c_i32), ("nnz", c_i64), ("row_ptr", c_vp),
                ("col_idx", c_vp), ("vals", c_vp)]


OPT_FIELDS = ["fp32_max_terms", "esc_max", "warp_max_ip", "block_max_ip", "warp_max_nnz",
              "block_max_nnz", "panel_cols", "row_cache_mb", "dense_splits",
              "stage_b", "narrow_warps", "narrow_max_ip", "hash_load_pct"]


class OptsStruct(ctypes.Structure):
    _fields_ = [(n, c_i32) for n in OPT_FIELDS] + [("reserved", c_i32 * 3)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_int, c_vp, c_i64, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp))

_P = ctypes.POINTER
_CSR = _P(CsrStruct)

PROTOTYPES = {
    "spgemm_opts_default": (ctypes.c_int, [_P(OptsStruct)]),
    "spgemm_plan_create": (ctypes.c_int, [_P(c_vp), _P(OptsStruct), ctypes.c_int]),
    "spgemm_plan_destroy": (ctypes.c_int, [c_vp]),
    "spgemm_workspace_bytes": (ctypes.c_int, [c_vp, _CSR, _CSR, _P(c_sz)]),
    "spgemm_workspace_init": (ctypes.c_int, [c_vp, c_vp, c_sz, c_vp]),
    "spgemm_count": (ctypes.c_int, [c_vp, _CSR, _CSR, c_vp, c_sz, c_vp, _P(c_i64), c_vp]),
    "spgemm_group": (ctypes.c_int, [c_vp, c_vp, c_i32, c_vp, c_i32, c_vp, c_sz, c_vp, c_vp, c_vp]),
    "spgemm_symbolic": (ctypes.c_int, [c_vp, _CSR, _CSR, c_vp, c_vp, c_sz, c_vp, _P(c_i64), c_vp]),
    "spgemm_row_ptr": (ctypes.c_int, [c_vp, c_vp, c_i32, c_vp, c_sz, c_vp, _P(c_i64), c_vp]),
    "spgemm_row_ptr_static": (ctypes.c_int, [c_vp, c_vp, c_i32, c_vp, _P(c_i64), c_vp]),
    "spgemm_numeric": (ctypes.c_int, [c_vp, _CSR, _CSR, c_vp, c_i32, c_i32, c_vp, c_vp, c_sz, c_vp,
                                      c_vp, c_vp]),
    "spgemm": (ctypes.c_int, [c_vp, _CSR, _CSR, c_vp, c_sz, c_vp, c_vp, c_vp, ALLOC_FN, c_vp,
                              _P(c_i64), c_vp]),
    "spgemm_backward_workspace_bytes": (ctypes.c_int, [c_vp, _CSR, _CSR, _P(c_sz)]),
    "spgemm_backward": (ctypes.c_int, [c_vp, _CSR, _CSR, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp, c_vp,
                                       c_sz, c_vp]),
    "spgemm_batched": (ctypes.c_int, [c_vp, _CSR, _CSR, c_vp, c_sz, c_vp, c_vp, c_vp, c_vp, c_vp,
                                      c_i64, c_vp, c_vp]),
    "spgemm_mcl_step": (ctypes.c_int, [c_vp, _CSR, ctypes.c_float, c_i32, ctypes.c_float, c_i32,
                                       c_vp, c_sz, c_vp, c_vp, c_vp, _P(c_i64), c_vp]),
    "spgemm_topk_dense": (ctypes.c_int, [c_vp, c_vp, c_i32, c_i32, c_i64, c_i32, c_vp, c_vp, c_vp,
                                         c_vp]),
    "spgemm_csr_scatter_dense": (ctypes.c_int, [c_vp, _CSR, c_vp, c_vp, c_i64, c_vp, c_sz, c_vp]),
    "spgemm_csr_gather_dense": (ctypes.c_int, [c_vp, _CSR, c_vp, c_i64, c_vp, c_vp, c_sz, c_vp]),
    "spgemm_sample_rows": (ctypes.c_int, [c_vp, _CSR, c_i32, c_vp, c_i32, c_vp, c_sz, c_vp, c_vp,
                                          c_vp, _P(c_i64), c_vp]),
    "spgemm_select_columns": (ctypes.c_int, [c_vp, _CSR, c_vp, c_sz, c_vp, c_vp, c_vp, c_vp, c_vp,
                                             c_vp, _P(c_i64), c_vp]),
    "spgemm_dense_gemm_workspace_bytes": (ctypes.c_int, [c_vp, c_i32, c_i32, c_i32, _P(c_sz)]),
    "spgemm_dense_gemm": (ctypes.c_int, [c_vp, c_i32, c_i32, c_i32, c_vp, c_i64, c_i32, c_vp, c_i64,
                                         c_i32, c_vp, c_i64, c_vp, c_sz, c_vp]),
    "spgemm_status": (ctypes.c_int, [c_vp, c_vp, c_vp, _P(ctypes.c_int)]),
    "spgemm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "spgemm_profile_enable": (ctypes.c_int, [c_vp, ctypes.c_int]),
    "spgemm_profile_read": (ctypes.c_int, [c_vp, _P(ctypes.c_double), _P(c_i64), ctypes.c_int]),
    "spgemm_kernel_count": (ctypes.c_int, []),
    "spgemm_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
    "spgemm_launch_total": (c_i64, [c_vp]),
}


def header_symbols() -> list[str]:
    """Every function declared in include/spgemm.h (parsed from the header text)."""
    here = os.path.dirname(os.path.abspath(__file__))
    txt = open(os.path.join(os.path.dirname(here), "include", "spgemm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(spgemm\w*)\s*\(", txt)))


def lib():
    """Load (building first if needed) and return the ctypes handle."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in PROTOTYPES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class SpgemmError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().spgemm_status_string(code).decode()
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


def check(code: int, where: str) -> None:
    if code != OK:
        raise SpgemmError(code, where)
