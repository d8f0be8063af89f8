"""Reference for the graph contraction S^T * A * S (Algorithm 7) computed
without any SpGEMM: with one 1.0 per row of S (row i in cluster label[i]),
(S^T A S)[c, c'] is the sum of A's entries (i, j) with label[i] = c and
label[j] = c', so the product is A's entries scattered by their labels.
Used by the contraction parity tests beside the oracle's per-product
comparison."""
import numpy as np


def label_scatter(A, labels: np.ndarray, m: int):
    """(row_ptr int64, col int32, val fp64, abs_sum fp64) of the m x m matrix
    whose entry (c, c') sums A's entries with labels (c, c'); abs_sum sums
    their magnitudes (the scale of the two-product error bound)."""
    rows = np.repeat(np.arange(A.rows, dtype=np.int64), np.diff(A.row_ptr.astype(np.int64)))
    key = labels[rows].astype(np.int64) * m + labels[A.col.astype(np.int64)]
    order = np.argsort(key, kind="stable")
    key = key[order]
    v = A.val[order].astype(np.float64)
    if key.size == 0:
        return np.zeros(m + 1, np.int64), np.zeros(0, np.int32), np.zeros(0), np.zeros(0)
    first = np.ones(key.size, dtype=bool)
    first[1:] = key[1:] != key[:-1]
    starts = np.flatnonzero(first)
    uk = key[starts]
    val = np.add.reduceat(v, starts)
    absum = np.add.reduceat(np.abs(v), starts)
    r = uk // m
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=m), out=row_ptr[1:])
    return row_ptr, (uk % m).astype(np.int32), val, absum


def assignment_labels(S) -> np.ndarray:
    """Cluster label of every row of an assignment matrix (one entry per row)."""
    assert np.array_equal(np.diff(S.row_ptr.astype(np.int64)), np.ones(S.rows, np.int64))
    return S.col.astype(np.int64)
