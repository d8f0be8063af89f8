"""Pins for the CPU oracle: it is checked against things other than itself
(hand-worked fixtures, dense numpy/scipy/torch arithmetic, closed forms,
algebraic identities, brute force), so that a dropped term, a wrong index or
a transposed operand in it fails here."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2512_12036_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _csr(d):
    return gen.HostCSR(d["rows"], d["cols"], np.array(d["row_ptr"], np.int32),
                       np.array(d["col"], np.int32), np.array(d["val"], np.float32))


def dense(A):
    """Dense fp64 copy with repeated entries summed (np.add.at, no oracle code)."""
    D = np.zeros((A.rows, A.cols))
    r = np.repeat(np.arange(A.rows), np.diff(A.row_ptr.astype(np.int64)))
    np.add.at(D, (r, A.col.astype(np.int64)), A.val.astype(np.float64))
    return D


def pattern(A):
    """Dense count of stored entries per position (explicit zeros count)."""
    D = np.zeros((A.rows, A.cols), dtype=np.int64)
    r = np.repeat(np.arange(A.rows), np.diff(A.row_ptr.astype(np.int64)))
    np.add.at(D, (r, A.col.astype(np.int64)), 1)
    return D


def absdense(A):
    D = np.zeros((A.rows, A.cols))
    r = np.repeat(np.arange(A.rows), np.diff(A.row_ptr.astype(np.int64)))
    np.add.at(D, (r, A.col.astype(np.int64)), np.abs(A.val.astype(np.float64)))
    return D


def oracle_dense(C):
    D = np.zeros((C.rows, C.cols))
    r = np.repeat(np.arange(C.rows), np.diff(C.row_ptr))
    D[r, C.col] = C.val
    return D


CASES = [
    dict(m=17, k=13, n=19, da=0.2, db=0.25, seed=1),
    dict(m=40, k=40, n=40, da=0.1, db=0.1, seed=2, duplicates=True),
    dict(m=31, k=7, n=50, da=0.5, db=0.3, seed=3, unsorted=True),
    dict(m=25, k=30, n=9, da=0.15, db=0.6, seed=4, explicit_zeros=0.3, signed=True),
    dict(m=1, k=1, n=1, da=1.0, db=1.0, seed=5),
    dict(m=64, k=64, n=64, da=0.05, db=0.05, seed=6),
]


def make(c):
    kw = {k: c[k] for k in ("duplicates", "unsorted", "explicit_zeros", "signed") if k in c}
    A = gen.random_csr(c["m"], c["k"], c["da"], c["seed"], **kw)
    B = gen.random_csr(c["k"], c["n"], c["db"], c["seed"] + 100, **kw)
    return A, B


def test_golden_hand_worked_product():
    g = json.load(open(os.path.join(GOLDEN, "gustavson_3x4x3.json")))
    A, B = _csr(g["A"]), _csr(g["B"])
    ip, total = oracle.ip_count(A, B)
    assert ip.tolist() == g["ip"] and total == sum(g["ip"])
    C = oracle.spgemm(A, B)
    assert C.row_ptr.tolist() == g["C"]["row_ptr"]
    assert C.col.tolist() == g["C"]["col"]
    assert C.val.tolist() == g["C"]["val"]
    assert C.bound.tolist() == g["C"]["bound"]


def test_golden_table1_grouping():
    g = json.load(open(os.path.join(GOLDEN, "table1_groups.json")))
    mp, off = oracle.group_rows(np.array(g["ip"]), g["thresholds"])
    assert mp.tolist() == g["map"]
    assert off.tolist() == g["offsets"]
    for grp in range(len(off) - 1):
        for r in mp[off[grp]:off[grp + 1]]:
            assert g["group"][r] == grp


@pytest.mark.parametrize("c", CASES)
def test_ip_count_against_brute_force(c):
    A, B = make(c)
    ip, total = oracle.ip_count(A, B)
    lenB = np.diff(B.row_ptr.astype(np.int64))
    brute = pattern(A) @ lenB                      # sum over stored (i,k) of |B_k|
    assert np.array_equal(ip, brute)
    colcount = np.bincount(A.col, minlength=A.cols)  # closed form for the total
    assert total == int(colcount @ lenB)


def test_ip_total_sum_of_squared_degrees():
    A = gen.erdos_renyi(300, 6, seed=9)
    _, total = oracle.ip_count(A, A)
    deg = np.diff(A.row_ptr.astype(np.int64))
    assert total == int((deg * deg).sum())


def test_group_rows_matches_stable_digitize():
    rng = np.random.default_rng(0)
    key = rng.integers(0, 20000, size=500)
    thr = [32, 512, 8192]
    mp, off = oracle.group_rows(key, thr)
    grp = np.digitize(key, thr)
    assert np.array_equal(mp, np.argsort(grp, kind="stable"))
    assert np.array_equal(np.diff(off), np.bincount(grp, minlength=4))


@pytest.mark.parametrize("c", CASES)
def test_symbolic_against_boolean_product(c):
    A, B = make(c)
    nnz = oracle.symbolic(A, B)
    want = ((pattern(A) @ pattern(B)) > 0).sum(axis=1)
    assert np.array_equal(nnz, want)


@pytest.mark.parametrize("c", CASES)
def test_numeric_against_dense_matmul(c):
    A, B = make(c)
    C = oracle.spgemm(A, B)
    struct = (pattern(A) @ pattern(B)) > 0
    r = np.repeat(np.arange(C.rows), np.diff(C.row_ptr))
    got = np.zeros(struct.shape, dtype=bool)
    got[r, C.col] = True
    assert np.array_equal(got, struct)
    for i in range(C.rows):                                   # sorted, no repeats
        cols = C.col[C.row_ptr[i]:C.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
    Dc = dense(A) @ dense(B)
    assert np.allclose(oracle_dense(C), Dc, rtol=1e-12, atol=1e-12)
    Db = absdense(A) @ absdense(B)
    assert np.allclose(C.bound, Db[r, C.col], rtol=1e-12, atol=0)
    assert np.all(np.abs(C.val) <= C.bound * (1 + 1e-12))


@pytest.mark.parametrize("c", CASES[:4])
def test_numeric_against_scipy(c):
    A, B = make(c)
    C = oracle.spgemm(A, B)
    SA = sp.csr_matrix((A.val.astype(np.float64), A.col, A.row_ptr), shape=(A.rows, A.cols))
    SB = sp.csr_matrix((B.val.astype(np.float64), B.col, B.row_ptr), shape=(B.rows, B.cols))
    assert np.allclose(oracle_dense(C), (SA @ SB).toarray(), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("c", CASES)
def test_transpose_identity(c):
    A, B = make(c)
    C = oracle.spgemm(A, B)
    Ct = oracle.spgemm(gen.transpose_structure(B), gen.transpose_structure(A))
    Cd = oracle_dense(C)
    Ctd = oracle_dense(Ct)
    assert np.allclose(Cd.T, Ctd, rtol=1e-12, atol=1e-12)
    assert C.nnz == Ct.nnz


@pytest.mark.parametrize("c", CASES)
def test_associativity_with_vector(c):
    A, B = make(c)
    C = oracle.spgemm(A, B)
    x = np.random.default_rng(c["seed"]).standard_normal(B.cols)
    SC = sp.csr_matrix((C.val, C.col, C.row_ptr), shape=(C.rows, C.cols))
    SA = sp.csr_matrix((A.val.astype(np.float64), A.col, A.row_ptr), shape=(A.rows, A.cols))
    SB = sp.csr_matrix((B.val.astype(np.float64), B.col, B.row_ptr), shape=(B.rows, B.cols))
    assert np.allclose(SC @ x, SA @ (SB @ x), rtol=1e-10, atol=1e-12)


def test_identity_and_permutation():
    B = gen.random_csr(30, 45, 0.2, seed=7, duplicates=True, unsorted=True)
    eye = gen.HostCSR(30, 30, np.arange(31, dtype=np.int32), np.arange(30, dtype=np.int32),
                      np.ones(30, np.float32))
    C = oracle.spgemm(eye, B)
    assert np.array_equal(oracle_dense(C), dense(B))
    assert np.array_equal(np.diff(C.row_ptr), (pattern(B) > 0).sum(axis=1))
    perm = np.random.default_rng(1).permutation(30)
    P = gen.HostCSR(30, 30, np.arange(31, dtype=np.int32), perm.astype(np.int32),
                    np.ones(30, np.float32))
    assert np.array_equal(oracle_dense(oracle.spgemm(P, B)), dense(B)[perm])


def test_edge_cases():
    empty = gen.HostCSR(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    B = gen.random_csr(5, 6, 0.5, seed=3)
    C = oracle.spgemm(empty, B)
    assert C.rows == 0 and C.nnz == 0
    Z = gen.HostCSR(4, 5, np.zeros(5, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    C = oracle.spgemm(Z, B)
    assert C.nnz == 0 and C.row_ptr.tolist() == [0] * 5
    dense_row = gen.HostCSR(1, 5, np.array([0, 5], np.int32), np.arange(5, dtype=np.int32),
                            np.ones(5, np.float32))
    C = oracle.spgemm(dense_row, B)
    assert np.allclose(oracle_dense(C), dense(dense_row) @ dense(B))
    bad = gen.HostCSR(2, 5, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32),
                      np.ones(2, np.float32))
    Bbad = gen.HostCSR(5, 3, np.array([0, 1, 1, 1, 1, 1], np.int32), np.array([7], np.int32),
                       np.ones(1, np.float32))
    with pytest.raises(ValueError):
        oracle.spgemm(bad, Bbad)


def test_row_subset_matches_full():
    A = gen.erdos_renyi(200, 8, seed=11)
    C = oracle.spgemm(A, A)
    rows = np.array([5, 0, 199, 77, 77], np.int32)
    S = oracle.spgemm(A, A, rows=rows)
    for q, i in enumerate(rows):
        a = slice(C.row_ptr[i], C.row_ptr[i + 1])
        b = slice(S.row_ptr[q], S.row_ptr[q + 1])
        assert np.array_equal(C.col[a], S.col[b])
        assert np.array_equal(C.val[a], S.val[b])


def test_contraction_sums_over_clusters():
    # S^T A S with S an assignment matrix (Alg. 7): entry (p, q) is the sum of
    # A over the pairs (i, j) with cluster(i) = p, cluster(j) = q, stored
    # exactly where such a pair holds a stored entry of A (explicit zeros
    # too), and the total of A is preserved. Small-integer values keep every
    # sum exact in fp32 and fp64, so the chain S^T A -> fp32 -> (S^T A) S is
    # compared exactly against a cluster-label scatter.
    A = gen.rmat_symmetric(10, 8, seed=4)
    vals = np.random.default_rng(6).integers(0, 9, size=A.col.size).astype(np.float32)
    A = gen.HostCSR(A.rows, A.cols, A.row_ptr, A.col, vals)
    m = 40
    S = gen.assignment_matrix(A.rows, m, seed=5)
    lab = S.col.astype(np.int64)
    T = oracle.spgemm(gen.transpose_structure(S), A)
    Th = gen.HostCSR(T.rows, T.cols, T.row_ptr.astype(np.int32), T.col,
                     T.val.astype(np.float32))
    C = oracle.spgemm(Th, S)
    r = np.repeat(np.arange(A.rows), np.diff(A.row_ptr.astype(np.int64)))
    D = np.zeros((m, m))
    np.add.at(D, (lab[r], lab[A.col]), vals.astype(np.float64))
    P = np.zeros((m, m), dtype=bool)
    P[lab[r], lab[A.col]] = True
    assert np.array_equal(oracle_dense(C), D)
    assert np.array_equal(np.diff(C.row_ptr), P.sum(axis=1))
    Cr = np.repeat(np.arange(C.rows), np.diff(C.row_ptr))
    assert P[Cr, C.col].all()
    assert C.val.sum() == float(vals.astype(np.float64).sum())


def test_block_diagonal_is_per_block_products():
    # rows of C depend only on their own row of A: the product of two
    # block-diagonal operands is the block-diagonal of the per-block products,
    # column offsets included, bit for bit (same terms in the same order)
    A1, B1 = gen.random_csr(30, 40, 0.2, seed=21), gen.random_csr(40, 50, 0.15, seed=22)
    A2, B2 = gen.random_csr(20, 35, 0.25, seed=23), gen.random_csr(35, 60, 0.1, seed=24)

    def sp_of(X):
        return sp.csr_matrix((X.val, X.col, X.row_ptr), shape=(X.rows, X.cols))

    def host_of(M):
        M = sp.csr_matrix(M)
        M.sort_indices()
        return gen.HostCSR(M.shape[0], M.shape[1], M.indptr.astype(np.int32),
                           M.indices.astype(np.int32), M.data.astype(np.float32))

    A = host_of(sp.block_diag([sp_of(A1), sp_of(A2)], format="csr"))
    B = host_of(sp.block_diag([sp_of(B1), sp_of(B2)], format="csr"))
    C = oracle.spgemm(A, B)
    for (r0, c0), Cb in (((0, 0), oracle.spgemm(A1, B1)), ((30, 50), oracle.spgemm(A2, B2))):
        for i in range(Cb.rows):
            a = slice(C.row_ptr[r0 + i], C.row_ptr[r0 + i + 1])
            b = slice(Cb.row_ptr[i], Cb.row_ptr[i + 1])
            assert np.array_equal(C.col[a], Cb.col[b] + c0)
            assert np.array_equal(C.val[a], Cb.val[b])
            assert np.array_equal(C.bound[a], Cb.bound[b])


def test_thread_count_does_not_change_result():
    A = gen.rmat_symmetric(10, 8, seed=3)
    C1 = oracle.spgemm(A, A, nthreads=1)
    C4 = oracle.spgemm(A, A, nthreads=4)
    assert np.array_equal(C1.row_ptr, C4.row_ptr)
    assert np.array_equal(C1.col, C4.col)
    assert np.array_equal(C1.val, C4.val)


@pytest.mark.parametrize("c", CASES[:4])
def test_backward_against_torch_autograd(c):
    torch = pytest.importorskip("torch")
    A, B = make(c)
    C = oracle.spgemm(A, B)
    rng = np.random.default_rng(c["seed"] + 7)
    dC = rng.standard_normal(C.nnz)
    dA, dB = oracle.backward(A, B, C, dC)
    G = np.zeros((C.rows, C.cols))
    r = np.repeat(np.arange(C.rows), np.diff(C.row_ptr))
    G[r, C.col] = dC
    DA = torch.tensor(dense(A), requires_grad=True)
    DB = torch.tensor(dense(B), requires_grad=True)
    (torch.tensor(G) * (DA @ DB)).sum().backward()
    ra = np.repeat(np.arange(A.rows), np.diff(A.row_ptr.astype(np.int64)))
    rb = np.repeat(np.arange(B.rows), np.diff(B.row_ptr.astype(np.int64)))
    assert np.allclose(dA, DA.grad.numpy()[ra, A.col], rtol=1e-10, atol=1e-12)
    assert np.allclose(dB, DB.grad.numpy()[rb, B.col], rtol=1e-10, atol=1e-12)


def test_backward_against_finite_differences():
    A = gen.random_csr(6, 5, 0.4, seed=21, signed=True)
    B = gen.random_csr(5, 7, 0.4, seed=22, signed=True)
    C = oracle.spgemm(A, B)
    dC = np.random.default_rng(3).standard_normal(C.nnz)
    dA, dB = oracle.backward(A, B, C, dC)
    G = np.zeros((C.rows, C.cols))
    G[np.repeat(np.arange(C.rows), np.diff(C.row_ptr)), C.col] = dC
    DA, DB = dense(A), dense(B)
    h = 1e-6
    ra = np.repeat(np.arange(A.rows), np.diff(A.row_ptr.astype(np.int64)))
    for j in range(A.nnz):
        E = np.zeros_like(DA)
        E[ra[j], A.col[j]] = h
        fd = ((G * ((DA + E) @ DB)).sum() - (G * ((DA - E) @ DB)).sum()) / (2 * h)
        assert abs(fd - dA[j]) < 1e-6
    rb = np.repeat(np.arange(B.rows), np.diff(B.row_ptr.astype(np.int64)))
    for t in range(B.nnz):
        E = np.zeros_like(DB)
        E[rb[t], B.col[t]] = h
        fd = ((G * (DA @ (DB + E))).sum() - (G * (DA @ (DB - E))).sum()) / (2 * h)
        assert abs(fd - dB[t]) < 1e-6


@pytest.mark.parametrize("order", [0, 1])
def test_mcl_step_against_brute_force(order):
    rng = np.random.default_rng(4 + order)
    M = gen.random_csr(40, 40, 0.4, seed=31 + order)
    M.val[:] = (rng.random(M.nnz) * 0.01).astype(np.float32)   # many below theta
    k, r = 5, 2.0
    # row 0 holds one value whose (inflated, for order 1) fp32 decision value
    # equals theta exactly: values below theta are removed, that one stays
    s0 = slice(M.row_ptr[0], M.row_ptr[1])
    assert M.row_ptr[1] - M.row_ptr[0] >= 3
    if order == 0:
        theta = float(np.float32(2e-3))
        edge = np.float32(theta)
    else:
        edge = np.float32(0.05)
        theta = float(np.float32(np.float64(edge) ** r))
    row0 = np.full(M.row_ptr[1] - M.row_ptr[0], 1e-4, np.float32)
    row0[0], row0[1] = edge, np.float32(0.08)
    M.val[s0] = row0
    out = oracle.mcl_step(M, theta, k, r, order)
    assert M.col[M.row_ptr[0]] in out.col[out.row_ptr[0]:out.row_ptr[1]].tolist()
    for i in range(M.rows):
        cols, vals = M.row(i)
        dec = vals if order == 0 else (vals.astype(np.float64) ** r).astype(np.float32)
        cand = [(float(dv), int(c), float(v)) for dv, c, v in zip(dec, cols, vals)
                if dv >= np.float32(theta)]
        cand.sort(key=lambda t: (-t[0], t[1]))
        keep = sorted(cand[:k], key=lambda t: t[1])
        s = slice(out.row_ptr[i], out.row_ptr[i + 1])
        assert out.col[s].tolist() == [c for _, c, _ in keep]
        w = np.array([v ** r for _, _, v in keep])
        if len(keep):
            assert np.allclose(out.val[s], w / w.sum(), rtol=1e-12)
            assert abs(out.val[s].sum() - 1.0) < 1e-12
        assert len(keep) <= k


def test_row_normalise():
    M = gen.random_csr(20, 20, 0.3, seed=41)
    out = oracle.row_normalise(M)
    r = np.repeat(np.arange(M.rows), np.diff(M.row_ptr.astype(np.int64)))
    sums = np.bincount(r, weights=out, minlength=M.rows)
    nonempty = np.diff(M.row_ptr) > 0
    assert np.allclose(sums[nonempty], 1.0, rtol=1e-14)
