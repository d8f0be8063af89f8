"""Host-side checks of the seeded input generators and of the row-block
planner (no GPU): every generated matrix is a valid CSR with the structure
its docstring promises, and the same seed gives the same matrix."""
import numpy as np
import pytest
import torch

from paper_2512_12036_gb300 import gen
from paper_2512_12036_gb300.api import split_rows


def dense(A: gen.HostCSR) -> np.ndarray:
    D = np.zeros((A.rows, A.cols))
    for i in range(A.rows):
        s, e = A.row_ptr[i], A.row_ptr[i + 1]
        D[i, A.col[s:e]] += A.val[s:e]
    return D


def assert_valid(A: gen.HostCSR, sorted_unique: bool = True):
    assert A.row_ptr.dtype == np.int32 and A.col.dtype == np.int32 and A.val.dtype == np.float32
    assert A.row_ptr.shape == (A.rows + 1,) and A.row_ptr[0] == 0
    assert (np.diff(A.row_ptr.astype(np.int64)) >= 0).all()
    assert A.row_ptr[-1] == A.col.size == A.val.size
    if A.col.size:
        assert A.col.min() >= 0 and A.col.max() < A.cols
    if sorted_unique:
        for i in range(A.rows):
            c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
            assert (np.diff(c) > 0).all()


def test_erdos_renyi_valid_and_seeded():
    A = gen.erdos_renyi(500, 8.0, seed=4)
    assert_valid(A)
    B = gen.erdos_renyi(500, 8.0, seed=4)
    assert (A.col == B.col).all() and (A.val == B.val).all()
    assert 6.0 < A.nnz / A.rows < 10.0
    assert (A.val > 0).all() and (A.val <= 1).all()


def test_rmat_symmetric_structure():
    A = gen.rmat_symmetric(10, 8, seed=2)
    assert_valid(A)
    D = dense(A) != 0
    assert (D == D.T).all()                         # symmetric pattern
    assert not D.diagonal().any()                   # no self-loops
    deg = D.sum(1)
    assert deg.max() > 8 * deg.mean()               # skewed degrees


def test_assignment_matrix_one_per_row():
    S = gen.assignment_matrix(1000, 37, seed=3)
    assert_valid(S)
    assert (np.diff(S.row_ptr) == 1).all() and (S.val == 1.0).all()
    assert S.cols == 37 and np.unique(S.col).size == 37


def test_transpose_structure_is_transpose():
    A = gen.random_csr(40, 25, 0.2, seed=5)
    T = gen.transpose_structure(A)
    assert_valid(T)
    assert np.array_equal(dense(T), dense(A).T)


def test_csr_from_coo_sorts_rows():
    r = np.array([2, 0, 2, 1, 0])
    c = np.array([3, 4, 0, 1, 2])
    v = np.arange(5, dtype=np.float32)
    A = gen.csr_from_coo(3, 5, r, c, v)
    assert_valid(A)
    assert list(A.col) == [2, 4, 1, 0, 3] and list(A.val) == [4, 1, 3, 2, 0]


def test_sample_rows_picks_strided_rows():
    A = gen.random_csr(103, 60, 0.1, seed=6)
    for stride in (1, 4, 10, 200):
        L = gen.sample_rows(A, stride)
        assert_valid(L)
        assert np.array_equal(dense(L), dense(A)[::stride])
    with pytest.raises(ValueError):
        gen.sample_rows(A, 0)


def test_split_rows_respects_limit():
    rng = np.random.default_rng(7)
    counts = torch.from_numpy(rng.integers(0, 50, size=1000).astype(np.int32))
    for limit in (49, 100, 1000, 10**9):
        bounds = split_rows(counts, limit)
        assert bounds[0][0] == 0 and bounds[-1][1] == 1000
        for (a0, a1), (b0, _) in zip(bounds, bounds[1:]):
            assert a1 == b0 and a1 > a0
        sums = [int(counts[a:b].sum()) for a, b in bounds]
        assert max(sums) <= limit
        # at least the fewest blocks the limit allows; exactly that many, cut
        # evenly (no small remainder), whenever an even cut must fit
        need = -(-int(counts.sum()) // limit)
        assert len(bounds) >= need
        if int(counts.sum()) / need + int(counts.max()) <= limit:
            assert len(bounds) == need
            assert min(sums) >= int(counts.sum()) / need - int(counts.max())
    with pytest.raises(ValueError):
        split_rows(counts, 10)


def test_rmat_graph_exact_n():
    for n, d, seed in ((1000, 8.0, 1), (3000, 20.0, 2), (1025, 4.0, 3)):
        A = gen.rmat_graph(n, d, seed=seed)
        assert A.rows == A.cols == n
        rows = np.repeat(np.arange(n), np.diff(A.row_ptr.astype(np.int64)))
        assert (A.col < n).all() and (A.col >= 0).all()
        assert not (rows == A.col).any()                     # no self-loops
        key = rows * n + A.col
        assert (np.diff(key) > 0).all()                      # sorted, no duplicates
        back = set(zip(A.col.tolist(), rows.tolist()))
        assert back == set(zip(rows.tolist(), A.col.tolist()))   # symmetric
        assert 0.5 * d <= A.nnz / n <= d                     # duplicates merged
        assert (A.val > 0).all() and (A.val <= 1).all()
        deg = np.diff(A.row_ptr)
        assert deg.max() > 4 * deg.mean()                    # skewed like R-MAT
    a, b = gen.rmat_graph(2000, 8, seed=5), gen.rmat_graph(2000, 8, seed=5)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.val, b.val)
