"""Property-based pins of the oracle (hypothesis draws the shapes, densities
and input conventions; CPU only, skipped where hypothesis is absent): on
every draw, against dense numpy arithmetic computed here,
  - structure: row i holds exactly the columns j with some stored (i,k) in
    A and stored (k,j) in B (the boolean product; stored zeros count),
    ascending and without repeats;
  - values: C = dense(A) @ dense(B) in fp64 (repeated entries summed);
  - error scale: bound = |A| @ |B| entry by entry;
  - counts: IP_i = sum over stored (i,k) of |B_k| (Alg. 1), nnz_i from the
    allocation phase equal to the row lengths of C."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
from paper_2512_12036_gb300 import gen  # noqa: E402


def dense(A, f=lambda v: v):
    D = np.zeros((A.rows, A.cols))
    r = np.repeat(np.arange(A.rows), np.diff(A.row_ptr.astype(np.int64)))
    np.add.at(D, (r, A.col.astype(np.int64)), f(A.val.astype(np.float64)))
    return D


def stored(A):
    D = np.zeros((A.rows, A.cols), dtype=bool)
    r = np.repeat(np.arange(A.rows), np.diff(A.row_ptr.astype(np.int64)))
    D[r, A.col.astype(np.int64)] = True
    return D


problems = st.fixed_dictionaries({
    "m": st.integers(0, 14), "k": st.integers(0, 14), "n": st.integers(0, 14),
    "da": st.floats(0.0, 1.0), "db": st.floats(0.0, 1.0),
    "seed": st.integers(0, 2**31 - 1),
    "duplicates": st.booleans(), "unsorted": st.booleans(),
    "explicit_zeros": st.sampled_from([0.0, 0.3]), "signed": st.booleans(),
})


def build(p):
    kw = {q: p[q] for q in ("duplicates", "unsorted", "explicit_zeros", "signed")}
    A = gen.random_csr(p["m"], p["k"], p["da"], p["seed"], **kw)
    B = gen.random_csr(p["k"], p["n"], p["db"], p["seed"] ^ 0x5A5A, **kw)
    return A, B


@settings(max_examples=150, deadline=None)
@given(problems)
def test_product_properties(p):
    A, B = build(p)
    C = oracle.spgemm(A, B)
    assert C.rows == A.rows and C.cols == B.cols
    S = (stored(A).astype(np.int64) @ stored(B).astype(np.int64)) > 0
    assert np.array_equal(np.diff(C.row_ptr), S.sum(axis=1))
    r = np.repeat(np.arange(C.rows), np.diff(C.row_ptr))
    assert S[r, C.col].all()
    for i in range(C.rows):
        seg = C.col[C.row_ptr[i]:C.row_ptr[i + 1]]
        assert (np.diff(seg) > 0).all()
    Cd = np.zeros((C.rows, C.cols))
    Cd[r, C.col] = C.val
    np.testing.assert_allclose(Cd, dense(A) @ dense(B), rtol=1e-12, atol=1e-12)
    Bd = np.zeros((C.rows, C.cols))
    Bd[r, C.col] = C.bound
    np.testing.assert_allclose(Bd, dense(A, np.abs) @ dense(B, np.abs), rtol=1e-12, atol=1e-12)


@settings(max_examples=150, deadline=None)
@given(problems)
def test_count_properties(p):
    A, B = build(p)
    ip, total = oracle.ip_count(A, B)
    blen = np.diff(B.row_ptr.astype(np.int64))
    want = np.array([blen[A.col[A.row_ptr[i]:A.row_ptr[i + 1]]].sum() for i in range(A.rows)],
                    dtype=np.int64)
    assert np.array_equal(np.asarray(ip, dtype=np.int64), want) and int(total) == int(want.sum())
    nnz = oracle.symbolic(A, B)
    S = (stored(A).astype(np.int64) @ stored(B).astype(np.int64)) > 0
    assert np.array_equal(np.asarray(nnz), S.sum(axis=1))
