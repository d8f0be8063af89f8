"""CPU oracle for the pruned GNN layer of Section IV-C (Eqs. 1-3).

TEST INFRASTRUCTURE ONLY (tests and the smoke check call it; the library
never imports it). Plain dense numpy / torch CPU arithmetic in fp64 on small
graphs, written from the equations:

  Eq. 2  TopK(X, k) = X (.) M_k, M_k[i, j] = 1 when X[i, j] is among the k
         largest values of row i ("per sample"). Values are compared as the
         fp32 numbers they are, in IEEE total order (a positive NaN above
         +inf, a negative NaN below -inf); equal values go to the smaller
         column (reading of "top-k values" for ties, which the paper leaves
         open).
  Eq. 1  X_l = A * TopK(X_{l-1}, k) * W_l.
  Eq. 3  dL/dX_{l-1} = M_k (.) (A^T * dL/dX_l * W_l^T); and, for the weight,
         dL/dW_l = (A * TopK(X_{l-1}, k))^T * dL/dX_l (the usual rule for a
         right factor, which Eq. 3 does not print).
"""
from __future__ import annotations

import numpy as np


def _order_key(x32: np.ndarray) -> np.ndarray:
    """uint64 key that orders fp32 values by IEEE total order."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    neg = (b & 0x80000000) != 0
    return np.where(neg, 0xFFFFFFFF - b, b | 0x80000000)


def topk_mask(X: np.ndarray, k: int) -> np.ndarray:
    """Boolean mask M_k of Eq. 2 for a dense fp32 matrix (n x d)."""
    X = np.asarray(X, dtype=np.float32)
    n, d = X.shape
    kk = max(0, min(k, d))
    M = np.zeros((n, d), dtype=bool)
    if kk == 0:
        return M
    key = _order_key(X)
    cols = np.arange(d)
    for i in range(n):
        # descending key, then ascending column
        order = np.lexsort((cols, 0xFFFFFFFF - key[i]))
        M[i, order[:kk]] = True
    return M


def topk_csr(X: np.ndarray, k: int):
    """TopK(X, k) as CSR arrays (row_ptr, col, val) in column order."""
    M = topk_mask(X, k)
    X = np.asarray(X, dtype=np.float32)
    rows, cols = np.nonzero(M)
    row_ptr = np.zeros(X.shape[0] + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr), cols.astype(np.int64), X[rows, cols]


def layer_forward(A: np.ndarray, X: np.ndarray, W: np.ndarray, k: int):
    """Eq. 1 in fp64: returns (Y, C, M) with C = A * TopK(X, k), Y = C * W."""
    M = topk_mask(X, k)
    T = np.where(M, np.asarray(X, dtype=np.float64), 0.0)
    C = np.asarray(A, dtype=np.float64) @ T
    return C @ np.asarray(W, dtype=np.float64), C, M


def layer_backward(A: np.ndarray, X: np.ndarray, W: np.ndarray, k: int, dY: np.ndarray):
    """Eq. 3 written out in fp64: returns (dX, dW)."""
    M = topk_mask(X, k)
    A64 = np.asarray(A, dtype=np.float64)
    W64 = np.asarray(W, dtype=np.float64)
    dY64 = np.asarray(dY, dtype=np.float64)
    T = np.where(M, np.asarray(X, dtype=np.float64), 0.0)
    dX = np.where(M, A64.T @ dY64 @ W64.T, 0.0)
    dW = (A64 @ T).T @ dY64
    return dX, dW


def layer_scales(A: np.ndarray, X: np.ndarray, W: np.ndarray, k: int, dY: np.ndarray):
    """Per-entry scales for tolerances: |A||T||W| for Y, |A|^T|dY||W|^T for
    dX and (|A||T|)^T |dY| for dW (fp64)."""
    M = topk_mask(X, k)
    aA = np.abs(np.asarray(A, dtype=np.float64))
    aT = np.where(M, np.abs(np.asarray(X, dtype=np.float64)), 0.0)
    aW = np.abs(np.asarray(W, dtype=np.float64))
    adY = np.abs(np.asarray(dY, dtype=np.float64))
    aC = aA @ aT
    return aC @ aW, aA.T @ adY @ aW.T, aC.T @ adY, aC
