"""Comparison helpers for the GPU-vs-oracle parity tests.

Acceptance (the value tolerance the library promises): row pointers and
sorted column indices identical to the oracle's; every value within
1e-5 * sum_k |a_ik||b_kj| of the oracle's fp64 value."""
import numpy as np

import oracle

REL_TOL = 1e-5


def compare(C_host, ref: oracle.OracleCSR, tol: float = REL_TOL, rows=None):
    """C_host: HostCSR from the GPU (row_ptr starting at 0). ref: oracle
    output for the same rows (all rows, or ``rows`` in that order)."""
    got_ptr = C_host.row_ptr.astype(np.int64)
    if rows is None:
        assert np.array_equal(got_ptr, ref.row_ptr), "row_ptr differs"
        assert np.array_equal(C_host.col, ref.col), "col differs"
        val = C_host.val
    else:
        cols, vals = [], []
        for i in rows:
            s, e = int(got_ptr[i]), int(got_ptr[i + 1])
            cols.append(C_host.col[s:e])
            vals.append(C_host.val[s:e])
        gnnz = np.array([c.size for c in cols])
        assert np.array_equal(gnnz, np.diff(ref.row_ptr)), "row nnz differs"
        col = np.concatenate(cols) if cols else np.zeros(0, np.int32)
        assert np.array_equal(col, ref.col), "col differs"
        val = np.concatenate(vals) if vals else np.zeros(0, np.float32)
    err = np.abs(val.astype(np.float64) - ref.val)
    lim = tol * ref.bound
    bad = err > lim
    if bad.any():
        q = int(np.argmax(err - lim))
        raise AssertionError(f"{int(bad.sum())} values outside tolerance; worst at {q}: "
                             f"got {val[q]!r} want {ref.val[q]!r} bound {ref.bound[q]!r}")
    return float((err / np.where(ref.bound > 0, ref.bound, 1)).max(initial=0.0))
