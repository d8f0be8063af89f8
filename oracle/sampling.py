"""CPU oracle for matrix-based bulk neighbourhood sampling (Section IV-C,
mini-batch training): P = Q^l * A, NORM, Q^{l-1} = SAMPLE(P, s) by inverse
transform sampling of s non-zeros per row, EXTRACT(A, Q^l, Q^{l-1}).

TEST INFRASTRUCTURE ONLY (the tests call it; the library never imports
it). Plain numpy in fp64, one row at a time:

  SAMPLE: a row with at most s entries keeps them all; otherwise each
  uniform u_t draws entry F^{-1}(u_t): mode 0 uniform over the entries
  (index floor(u * len)); mode 1 weights = max(value, 0); mode 2 weights =
  value^2; the draw is the first entry whose cumulative weight exceeds
  u * total (total 0: mode 0). The distinct drawn columns, ascending, value
  1. NORM is the division by the row total inside F (reading: the paper
  names NORM without fixing it; per row, inverse transform sampling on
  unnormalised weights is the same draw as on the normalised row).
  Column selection: the ascending distinct columns of Q^{l-1}.
  EXTRACT: the submatrix of A with Q^l's rows and Q^{l-1}'s selected columns.
"""
from __future__ import annotations

import numpy as np


def sample_rows(row_ptr, col, val, s: int, u: np.ndarray, mode: int):
    """Returns (row_ptr, col, val, gap): gap = the smallest distance of any
    weighted draw's u * total to a cumulative boundary, over total (inf if
    none), so a test can keep its draws clear of rounding ties."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col)
    val = np.asarray(val, dtype=np.float32)
    u = np.asarray(u, dtype=np.float32).reshape(len(rp) - 1, s)
    out_rows, gap = [], np.inf
    for i in range(len(rp) - 1):
        a, b = rp[i], rp[i + 1]
        n = b - a
        if n <= s:
            picks = col[a:b]
        else:
            w = val[a:b].astype(np.float64)
            w = w * w if mode == 2 else np.maximum(w, 0.0)
            total = float(w.sum()) if mode != 0 else 0.0
            picks = []
            for t in range(s):
                ut = float(u[i, t])
                if mode == 0 or not total > 0.0:
                    idx = min(n - 1, int(np.floor(ut * n)))
                else:
                    cum = np.cumsum(w)
                    target = ut * total
                    idx = int(np.searchsorted(cum, target, side="right"))
                    idx = min(idx, n - 1)
                    lo = cum[idx - 1] if idx > 0 else 0.0
                    gap = min(gap, (target - lo) / total, (cum[idx] - target) / total)
                picks.append(col[a + idx])
        out_rows.append(np.unique(np.asarray(picks, dtype=np.int64)))
    counts = np.array([r.size for r in out_rows], dtype=np.int64)
    out_rp = np.concatenate([[0], np.cumsum(counts)])
    out_col = np.concatenate(out_rows) if out_rows else np.zeros(0, np.int64)
    return out_rp, out_col, np.ones(out_col.size, np.float32), gap


def select_columns(col: np.ndarray, ncols: int):
    """(vertices, rank): the ascending distinct columns and, per column of
    the matrix, its rank among them (the exclusive prefix of the flags)."""
    vertices = np.unique(np.asarray(col, dtype=np.int64))
    flag = np.zeros(ncols, dtype=np.int64)
    flag[vertices] = 1
    rank = np.concatenate([[0], np.cumsum(flag)])
    return vertices, rank


def extract(A_dense: np.ndarray, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """EXTRACT: A restricted to the given rows and columns (dense)."""
    return A_dense[np.ix_(np.asarray(rows, dtype=np.int64), np.asarray(cols, dtype=np.int64))]
