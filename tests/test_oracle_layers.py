"""Pins of the pruned-GNN-layer oracle (Section IV-C, Eqs. 1-3) against
definitions computed another way: a plain Python sort for the top-k mask,
the unpruned product for k = d, torch autograd and finite differences for
the gradients."""
import math

import numpy as np
import pytest
import torch

from oracle import layers


def brute_topk_mask(X, k):
    """Sort every row by (-value, column) with Python's sort (finite values)."""
    n, d = X.shape
    M = np.zeros((n, d), dtype=bool)
    for i in range(n):
        order = sorted(range(d), key=lambda j: (-float(X[i, j]), j))
        for j in order[:max(0, min(k, d))]:
            M[i, j] = True
    return M


@pytest.mark.parametrize("k", [0, 1, 5, 16, 17, 40])
def test_topk_mask_matches_sort(k):
    rng = np.random.default_rng(3)
    X = rng.normal(size=(50, 17)).astype(np.float32)
    X[:10] = np.round(X[:10])            # many ties
    X[10:15] = 0.0
    X[X == 0] = 0.0                      # +0 only: a plain sort ties -0 with +0
    assert np.array_equal(layers.topk_mask(X, k), brute_topk_mask(X, k))
    M = layers.topk_mask(X, k)
    assert (M.sum(1) == min(k, 17)).all()


def test_topk_special_values():
    # IEEE total order: +NaN above +inf, -NaN below -inf, +0 above -0
    row = np.array([1.0, np.nan, -np.inf, 2.0, 0.0, -0.0, np.inf], dtype=np.float32)
    neg_nan = np.array([0xFFC00000], dtype=np.uint32).view(np.float32)[0]
    row = np.append(row, neg_nan).astype(np.float32)
    X = row[None, :]
    got = lambda k: set(np.nonzero(layers.topk_mask(X, k)[0])[0].tolist())  # noqa: E731
    assert got(1) == {1}
    assert got(2) == {1, 6}
    assert got(4) == {1, 6, 3, 0}
    assert got(5) == {1, 6, 3, 0, 4}
    assert got(6) == {1, 6, 3, 0, 4, 5}
    assert got(7) == {1, 6, 3, 0, 4, 5, 2}
    assert got(8) == set(range(8))


def test_topk_csr_layout():
    X = np.array([[3, 1, 2, 5], [0, 0, 0, 0], [-1, -2, -3, -4]], dtype=np.float32)
    rp, col, val = layers.topk_csr(X, 2)
    assert rp.tolist() == [0, 2, 4, 6]
    assert col.tolist() == [0, 3, 0, 1, 0, 1]
    assert val.tolist() == [3, 5, 0, 0, -1, -2]


def _problem(n=30, d=12, dout=7, seed=5):
    rng = np.random.default_rng(seed)
    A = (rng.random((n, n)) < 0.2) * rng.normal(size=(n, n))
    X = rng.normal(size=(n, d)).astype(np.float32)
    W = rng.normal(size=(d, dout))
    dY = rng.normal(size=(n, dout))
    return A, X, W, dY


def test_forward_without_pruning_is_plain_product():
    A, X, W, _ = _problem()
    Y, C, M = layers.layer_forward(A, X, W, k=X.shape[1])
    assert M.all()
    np.testing.assert_allclose(Y, A @ X.astype(np.float64) @ W, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(C, A @ X.astype(np.float64), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("k", [1, 4])
def test_forward_with_pruning_is_masked_product(k):
    # Eq. 1 with Eq. 2's mask taken from a plain Python sort of each row
    A, X, W, _ = _problem()
    Y, C, M = layers.layer_forward(A, X, W, k=k)
    Mb = brute_topk_mask(X, k)
    assert np.array_equal(M, Mb) and (M.sum(axis=1) == k).all()
    T = np.where(Mb, X.astype(np.float64), 0.0)
    np.testing.assert_allclose(C, A @ T, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Y, A @ T @ W, rtol=1e-12, atol=1e-12)


def test_backward_matches_autograd():
    A, X, W, dY = _problem()
    k = 4
    dX, dW = layers.layer_backward(A, X, W, k, dY)
    M = torch.from_numpy(layers.topk_mask(X, k))
    Xt = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    Wt = torch.tensor(W, dtype=torch.float64, requires_grad=True)
    Y = torch.from_numpy(A) @ (Xt * M) @ Wt
    Y.backward(torch.from_numpy(dY))
    np.testing.assert_allclose(dX, Xt.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dW, Wt.grad.numpy(), rtol=1e-12, atol=1e-12)
    assert (dX[~layers.topk_mask(X, k)] == 0).all()


def test_backward_matches_finite_differences():
    A, X, W, dY = _problem(n=12, d=6, dout=3, seed=8)
    k = 3
    dX, dW = layers.layer_backward(A, X, W, k, dY)
    M = layers.topk_mask(X, k)

    def loss(Xv, Wv):
        T = np.where(M, Xv, 0.0)       # the mask is held fixed (piecewise-linear)
        return float(((A @ T @ Wv) * dY).sum())

    X64 = X.astype(np.float64)
    eps = 1e-6
    for (i, j) in [tuple(p) for p in np.argwhere(M)[:6]]:
        Xp, Xm = X64.copy(), X64.copy()
        Xp[i, j] += eps
        Xm[i, j] -= eps
        fd = (loss(Xp, W) - loss(Xm, W)) / (2 * eps)
        assert math.isclose(fd, dX[i, j], rel_tol=1e-6, abs_tol=1e-8)
    for (i, j) in [(0, 0), (2, 1), (5, 2)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[i, j] += eps
        Wm[i, j] -= eps
        fd = (loss(X64, Wp) - loss(X64, Wm)) / (2 * eps)
        assert math.isclose(fd, dW[i, j], rel_tol=1e-6, abs_tol=1e-8)
