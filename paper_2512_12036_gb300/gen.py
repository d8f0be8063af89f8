"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module only builds matrices: graph structure plus random values. It
holds none of the SpGEMM arithmetic (no products, no accumulation, no
counting of intermediate products), so that the oracle and the kernels can
both consume its output without sharing any of the method.

Every generator is deterministic in its ``seed`` (numpy PCG64). Matrices come
back as :class:`HostCSR`: int32 row pointers and column indices, float32
values, rows sorted by column with no duplicates unless a generator says
otherwise.

Workload shapes follow the paper's evaluation (Section V and the matrix
table of Section VI): sparse graphs with 3-120 nonzeros per row and skewed
maximum row lengths, which the Erdos-Renyi and R-MAT families below stand in
for; the paper's SuiteSparse/SNAP/OGB matrices are not used.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class HostCSR:
    """CSR matrix on the host: row_ptr (rows+1, int32), col (nnz, int32), val (nnz, float32)."""

    rows: int
    cols: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def row(self, i: int):
        s, e = int(self.row_ptr[i]), int(self.row_ptr[i + 1])
        return self.col[s:e], self.val[s:e]


def csr_from_coo(rows: int, cols: int, r: np.ndarray, c: np.ndarray, v: np.ndarray,
                 sort: bool = True) -> HostCSR:
    """Assemble CSR from coordinate triples. With ``sort`` the entries are ordered
    by (row, col); duplicates are kept as separate entries (callers dedup first)."""
    r = np.asarray(r, dtype=np.int64)
    c = np.asarray(c, dtype=np.int64)
    v = np.asarray(v, dtype=np.float32)
    if sort and r.size:
        if cols > 0 and rows * cols < (1 << 62):
            order = np.argsort(r * cols + c, kind="stable")
        else:
            order = np.lexsort((c, r))
        r, c, v = r[order], c[order], v[order]
    counts = np.bincount(r, minlength=rows) if r.size else np.zeros(rows, dtype=np.int64)
    row_ptr = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return HostCSR(rows, cols, row_ptr.astype(np.int32), c.astype(np.int32),
                   np.ascontiguousarray(v, dtype=np.float32))


def uniform_open_closed(rng: np.random.Generator, n: int) -> np.ndarray:
    """float32 values in (0, 1]."""
    return (np.float32(1.0) - rng.random(n, dtype=np.float32)).astype(np.float32)


def _undirected_to_csr(n: int, u: np.ndarray, v: np.ndarray, w: np.ndarray,
                       self_loop_vals: np.ndarray | None = None) -> HostCSR:
    """Mirror unique undirected pairs u<v (one value per pair) into a symmetric CSR."""
    rr = np.concatenate([u, v])
    cc = np.concatenate([v, u])
    ww = np.concatenate([w, w])
    if self_loop_vals is not None:
        d = np.arange(n, dtype=np.int64)
        rr = np.concatenate([rr, d])
        cc = np.concatenate([cc, d])
        ww = np.concatenate([ww, self_loop_vals])
    return csr_from_coo(n, n, rr, cc, ww)


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + neighbour compare; faster here than
    numpy's hash-based unique on tens of millions of int64 keys)."""
    a = np.sort(a)
    if a.size == 0:
        return a
    keep = np.empty(a.size, dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def _unique_pairs(n: int, u: np.ndarray, v: np.ndarray):
    """Unique unordered pairs with u != v, returned as (lo, hi) sorted by key."""
    keep = u != v
    u, v = u[keep], v[keep]
    lo = np.minimum(u, v).astype(np.int64)
    hi = np.maximum(u, v).astype(np.int64)
    key = _sorted_unique(lo * n + hi)
    return key // n, key % n


def erdos_renyi(n: int, avg_degree: float, seed: int, self_loops: bool = False) -> HostCSR:
    """Symmetric G(n, p) adjacency with p = avg_degree / (n - 1), values U(0,1].

    The number of undirected edges is drawn from Binomial(n(n-1)/2, p) and that
    many distinct pairs are drawn uniformly, which is exactly G(n, p).
    """
    rng = np.random.default_rng(seed)
    if n <= 1:
        return csr_from_coo(n, n, np.zeros(0), np.zeros(0), np.zeros(0))
    pairs = n * (n - 1) // 2
    p = min(1.0, avg_degree / (n - 1))
    m_edges = int(rng.binomial(pairs, p))
    lo = np.zeros(0, dtype=np.int64)
    hi = np.zeros(0, dtype=np.int64)
    while lo.size < m_edges:
        need = m_edges - lo.size
        draw = int(need * 1.1) + 16
        u = rng.integers(0, n, size=draw, dtype=np.int64)
        v = rng.integers(0, n, size=draw, dtype=np.int64)
        nl, nh = _unique_pairs(n, np.concatenate([lo, u]), np.concatenate([hi, v]))
        if nl.size > m_edges:
            pick = np.sort(rng.choice(nl.size, size=m_edges, replace=False))
            nl, nh = nl[pick], nh[pick]
        lo, hi = nl, nh
    w = uniform_open_closed(rng, lo.size)
    loops = uniform_open_closed(rng, n) if self_loops else None
    return _undirected_to_csr(n, lo, hi, w, loops)


def rmat_edges(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
               permute: bool = True):
    """Directed R-MAT edge list (Chakrabarti et al. 2004): each of edge_factor*2^scale
    edges picks one quadrant per level with probabilities (a, b, c, d). Vertex labels
    are then permuted at random, as Graph500 does, so hubs are not clustered at low ids."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    ne = edge_factor * n
    u = np.zeros(ne, dtype=np.int64)
    v = np.zeros(ne, dtype=np.int64)
    ab = a + b
    abc = a + b + c
    for level in range(scale):
        r = rng.random(ne, dtype=np.float32)
        bit = np.int64(1) << (scale - 1 - level)
        right = ((r >= a) & (r < ab)) | (r >= abc)      # quadrants b and d: column bit set
        down = r >= ab                                   # quadrants c and d: row bit set
        u += down.astype(np.int64) * bit
        v += right.astype(np.int64) * bit
    if permute:
        perm = rng.permutation(n).astype(np.int64)
        u, v = perm[u], perm[v]
    return n, u, v, rng


def rmat_symmetric(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19,
                   c: float = 0.19, seed: int = 2, self_loops: bool = False) -> HostCSR:
    """Symmetrised, deduplicated R-MAT adjacency without self-loops (unless asked),
    values U(0,1] with one value per undirected edge."""
    n, u, v, rng = rmat_edges(scale, edge_factor, a, b, c, seed)
    lo, hi = _unique_pairs(n, u, v)
    w = uniform_open_closed(rng, lo.size)
    loops = uniform_open_closed(rng, n) if self_loops else None
    return _undirected_to_csr(n, lo, hi, w, loops)


def rmat_graph(n: int, avg_degree: float, seed: int, a: float = 0.57, b: float = 0.19,
               c: float = 0.19) -> HostCSR:
    """Symmetric R-MAT graph on exactly n vertices with about ``avg_degree``
    stored entries per row: n * avg_degree / 2 directed R-MAT edges at scale
    ceil(log2 n), every edge with an endpoint >= n drawn again (from the
    same generator) until all lie below n; then as rmat_symmetric (labels
    permuted, self-loops dropped, symmetrised, deduplicated, U(0,1] values)."""
    if n <= 1:
        return csr_from_coo(n, n, np.zeros(0), np.zeros(0), np.zeros(0))
    scale = max(1, int(np.ceil(np.log2(n))))
    rng = np.random.default_rng(seed)
    ne = max(1, int(round(n * avg_degree / 2)))
    ab, abc = a + b, a + b + c
    u = np.zeros(0, dtype=np.int64)
    v = np.zeros(0, dtype=np.int64)
    while u.size < ne:
        m = ne - u.size
        uu = np.zeros(m, dtype=np.int64)
        vv = np.zeros(m, dtype=np.int64)
        for level in range(scale):
            r = rng.random(m, dtype=np.float32)
            bit = np.int64(1) << (scale - 1 - level)
            uu += (r >= ab).astype(np.int64) * bit
            vv += (((r >= a) & (r < ab)) | (r >= abc)).astype(np.int64) * bit
        keep = (uu < n) & (vv < n)
        u = np.concatenate([u, uu[keep]])
        v = np.concatenate([v, vv[keep]])
    perm = rng.permutation(n).astype(np.int64)
    lo, hi = _unique_pairs(n, perm[u], perm[v])
    return _undirected_to_csr(n, lo, hi, uniform_open_closed(rng, lo.size))


def assignment_matrix(n: int, m: int, seed: int) -> HostCSR:
    """S (n x m): row r holds a single 1.0 at a uniformly drawn cluster id."""
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, m, size=n, dtype=np.int64)
    row_ptr = np.arange(n + 1, dtype=np.int32)
    return HostCSR(n, m, row_ptr, lab.astype(np.int32), np.ones(n, dtype=np.float32))


def random_csr(rows: int, cols: int, density: float, seed: int, *, duplicates: bool = False,
               unsorted: bool = False, explicit_zeros: float = 0.0,
               signed: bool = False) -> HostCSR:
    """Generic random sparse matrix for edge-case tests.

    ``duplicates`` repeats some entries inside a row, ``unsorted`` shuffles the
    entries of each row, ``explicit_zeros`` stores that fraction of entries with
    value 0.0, ``signed`` draws values from U(-1, 1) instead of U(0, 1]."""
    rng = np.random.default_rng(seed)
    nnz = int(round(rows * cols * density))
    if rows == 0 or cols == 0:
        nnz = 0
    r = rng.integers(0, max(rows, 1), size=nnz, dtype=np.int64)
    c = rng.integers(0, max(cols, 1), size=nnz, dtype=np.int64)
    key = _sorted_unique(r * max(cols, 1) + c)
    r, c = key // max(cols, 1), key % max(cols, 1)
    if duplicates and r.size:
        extra = rng.integers(0, r.size, size=max(1, r.size // 5))
        r = np.concatenate([r, r[extra]])
        c = np.concatenate([c, c[extra]])
    if signed:
        v = (rng.random(r.size) * 2 - 1).astype(np.float32)
    else:
        v = uniform_open_closed(rng, r.size)
    if explicit_zeros > 0 and r.size:
        v[rng.random(r.size) < explicit_zeros] = 0.0
    csr = csr_from_coo(rows, cols, r, c, v)
    if unsorted and csr.nnz:
        for i in range(rows):
            s, e = int(csr.row_ptr[i]), int(csr.row_ptr[i + 1])
            if e - s > 1:
                p = rng.permutation(e - s) + s
                csr.col[s:e] = csr.col[p]
                csr.val[s:e] = csr.val[p]
    return csr


def sample_rows(A: HostCSR, stride: int) -> HostCSR:
    """Rows 0, stride, 2*stride, ... of A (same columns): a smaller left
    operand with the row-length mix of the whole matrix."""
    if stride < 1:
        raise ValueError("stride must be >= 1")
    rp = A.row_ptr.astype(np.int64)
    pick = np.arange(0, A.rows, stride)
    lens = rp[pick + 1] - rp[pick]
    row_ptr = np.zeros(pick.size + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    idx = np.repeat(rp[pick] - row_ptr[:-1], lens) + np.arange(int(row_ptr[-1]))
    return HostCSR(int(pick.size), A.cols, row_ptr.astype(np.int32), A.col[idx].copy(),
                   A.val[idx].copy())


def transpose_structure(A: HostCSR) -> HostCSR:
    """Plain re-layout of A as A^T (no arithmetic on values)."""
    r = np.repeat(np.arange(A.rows, dtype=np.int64), np.diff(A.row_ptr.astype(np.int64)))
    return csr_from_coo(A.cols, A.rows, A.col.astype(np.int64), r, A.val)


# ---------------------------------------------------------------------------
# Batched GNN aggregation inputs: many small (A_hat_b, X_b) pairs.
# ---------------------------------------------------------------------------

@dataclass
class GNNBatch:
    """Independent subgraph problems, each C_b = A_hat_b @ X_b, concatenated.

    ``A`` and ``X`` are the block-diagonal stacks; ``node_off`` (num+1, int64)
    gives each subgraph's node range, which is both its row range in A/X and its
    column range in A. X's columns (features) are shared: X is (N x F)."""

    num: int
    node_off: np.ndarray
    A: HostCSR
    X: HostCSR
    features: int


def sym_normalised_adjacency(n: int, avg_degree: float, rng: np.random.Generator) -> HostCSR:
    """A_hat = D^-1/2 (A + I) D^-1/2 for an undirected ER graph (the GCN
    convention); input preparation for the aggregation C = A_hat X."""
    seed = int(rng.integers(0, 2**31 - 1))
    A = erdos_renyi(n, avg_degree, seed)
    r = np.repeat(np.arange(n, dtype=np.int64), np.diff(A.row_ptr.astype(np.int64)))
    c = A.col.astype(np.int64)
    r = np.concatenate([r, np.arange(n)])
    c = np.concatenate([c, np.arange(n)])
    deg = np.bincount(r, minlength=n).astype(np.float64)
    w = (1.0 / np.sqrt(deg[r] * deg[c])).astype(np.float32)
    return csr_from_coo(n, n, r, c, w)


def topk_rows(dense: np.ndarray, k: int) -> HostCSR:
    """Keep the k largest values of each row (ties to the smaller column index),
    as the pruned feature matrix TopK(X, k) = X * M_k of the GNN layer."""
    n, f = dense.shape
    k = min(k, f)
    order = np.lexsort((np.broadcast_to(np.arange(f), dense.shape), -dense), axis=1)[:, :k]
    cols = np.sort(order, axis=1)
    vals = np.take_along_axis(dense, cols, axis=1).astype(np.float32)
    row_ptr = (np.arange(n + 1, dtype=np.int64) * k).astype(np.int32)
    return HostCSR(n, f, row_ptr, cols.reshape(-1).astype(np.int32), vals.reshape(-1))


def _topk_columns(dense: np.ndarray, k: int) -> np.ndarray:
    """Ascending column indices of the k largest values of every row."""
    try:
        import torch
        idx = torch.topk(torch.from_numpy(dense), k, dim=1).indices.numpy()
    except ImportError:
        idx = np.argpartition(-dense, k - 1, axis=1)[:, :k]
    idx = np.sort(idx, axis=1)
    return idx


def gnn_batch(num: int, seed: int, n_min: int = 64, n_max: int = 2048, deg_min: float = 4.0,
              deg_max: float = 32.0, features: int = 256, k: int = 32,
              chunk_rows: int = 131072) -> GNNBatch:
    """``num`` subgraphs with n log-uniform in [n_min, n_max], average degree
    U[deg_min, deg_max], sym-normalised A_hat, and X = TopK(N(0,1), k) per row.

    Vectorised over all subgraphs: each graph draws its G(n, p) edge count
    from the binomial, candidate pairs are drawn uniformly inside every graph
    and deduplicated, and a uniformly random subset of the distinct pairs of
    the right size is kept per graph (redrawing for graphs left short)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=num)).astype(np.int64)
    sizes = np.clip(sizes, n_min, n_max)
    degs = rng.uniform(deg_min, deg_max, size=num)
    node_off = np.zeros(num + 1, dtype=np.int64)
    np.cumsum(sizes, out=node_off[1:])
    N = int(node_off[-1])
    pairs = sizes * (sizes - 1) // 2
    p = np.minimum(1.0, degs / np.maximum(sizes - 1, 1))
    want = rng.binomial(pairs, p).astype(np.int64)
    done_keys = []
    pending = np.arange(num)
    pend_keys = np.zeros(0, dtype=np.int64)
    have = np.zeros(num, dtype=np.int64)
    for _ in range(64):
        if pending.size == 0:
            break
        draw = (want[pending] - have[pending]) * 5 // 4 + 16
        g = np.repeat(pending, draw)
        n_g = sizes[g]
        u = (rng.random(g.size) * n_g).astype(np.int64)
        v = (rng.random(g.size) * n_g).astype(np.int64)
        ok = u != v
        g, u, v = g[ok], u[ok], v[ok]
        lo = np.minimum(u, v) + node_off[g]
        hi = np.maximum(u, v) + node_off[g]
        keys = _sorted_unique(np.concatenate([pend_keys, lo * N + hi]))
        graph_of = np.searchsorted(node_off, keys // N, side="right") - 1
        cnt = np.bincount(graph_of, minlength=num)
        have[pending] = cnt[pending]
        full = cnt[graph_of] >= want[graph_of]
        # graphs with enough distinct pairs: keep a uniformly random subset
        fk, fg = keys[full], graph_of[full]
        prio = rng.integers(0, 1 << 31, size=fk.size, dtype=np.int64)
        order = np.argsort(fg * (1 << 31) + prio, kind="stable")
        fk, fg = fk[order], fg[order]
        first = np.searchsorted(fg, np.arange(num))
        rank = np.arange(fk.size) - first[fg]
        done_keys.append(fk[rank < want[fg]])
        pend_keys = keys[~full]
        pending = pending[have[pending] < want[pending]]
    keys = np.concatenate(done_keys) if done_keys else np.zeros(0, dtype=np.int64)
    lo, hi = keys // N, keys % N
    ids = np.arange(N, dtype=np.int64)
    full = np.sort(np.concatenate([lo * N + hi, hi * N + lo, ids * N + ids]))
    r, c = full // N, full % N
    deg = np.bincount(r, minlength=N).astype(np.float64)
    w = (1.0 / np.sqrt(deg[r] * deg[c])).astype(np.float32)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=N), out=row_ptr[1:])
    A = HostCSR(N, N, row_ptr.astype(np.int32), c.astype(np.int32), w)
    kk = min(k, features)
    xcols = np.empty((N, kk), dtype=np.int32)
    xvals = np.empty((N, kk), dtype=np.float32)
    for r0 in range(0, N, chunk_rows):
        r1 = min(N, r0 + chunk_rows)
        dense = rng.standard_normal((r1 - r0, features), dtype=np.float32)
        top = _topk_columns(dense, kk)
        xcols[r0:r1] = top
        xvals[r0:r1] = np.take_along_axis(dense, top, axis=1)
    X = HostCSR(N, features, (np.arange(N + 1, dtype=np.int64) * kk).astype(np.int32),
                xcols.reshape(-1), xvals.reshape(-1))
    return GNNBatch(num, node_off, A, X, features)
