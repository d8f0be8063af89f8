"""The label-scatter reference of the contraction S^T*A*S (tests/contraction.py)
against dense fp64 matrix products on small inputs (no GPU)."""
import numpy as np

from contraction import assignment_labels, label_scatter
from paper_2512_12036_gb300 import gen


def dense(M):
    D = np.zeros((M.rows, M.cols))
    rows = np.repeat(np.arange(M.rows), np.diff(M.row_ptr.astype(np.int64)))
    np.add.at(D, (rows, M.col), M.val.astype(np.float64))
    return D


def test_label_scatter_is_St_A_S():
    for seed, n, m in ((1, 60, 7), (2, 200, 31), (3, 5, 5)):
        A = gen.random_csr(n, n, 0.08, seed=seed, signed=True) if n > 5 else \
            gen.random_csr(n, n, 0.5, seed=seed)
        S = gen.assignment_matrix(n, m, seed=seed + 10)
        want = dense(S).T @ dense(A) @ dense(S)
        rp, col, val, absum = label_scatter(A, assignment_labels(S), m)
        got = np.zeros((m, m))
        struct = np.zeros((m, m), dtype=bool)
        rows = np.repeat(np.arange(m), np.diff(rp))
        got[rows, col] = val
        struct[rows, col] = True
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
        # structure: a cluster pair is stored iff some stored entry of A maps to it
        Ab = dense_struct(A)
        assert np.array_equal(struct, (dense(S).T @ Ab @ dense(S)) > 0)
        assert (absum >= np.abs(val) - 1e-12).all()


def dense_struct(M):
    D = np.zeros((M.rows, M.cols), dtype=bool)
    rows = np.repeat(np.arange(M.rows), np.diff(M.row_ptr.astype(np.int64)))
    D[rows, M.col] = True
    return D
