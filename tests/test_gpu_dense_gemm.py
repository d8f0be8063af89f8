"""The dense fp32 GEMM of the pruned GNN layer (spgemm_dense_gemm) against
fp64 numpy products: every transpose combination, ragged edges (sizes that
are not multiples of the 128 x 128 tile or the k-step of 16), leading
dimensions that rule out vector loads, a long reduction split over blocks
along K (with and without the workspace), and K = 0. Bound: an fp32 sum of
K fused products is within gamma_K * sum |a||b| of the exact value
(gamma_K = K * 2^-24); a split reduction is within the bound of its longest
piece plus fp64 rounding."""
import numpy as np
import pytest
import torch

from paper_2512_12036_gb300 import Plan, _lib, gnn

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


@pytest.fixture(scope="module")
def plan():
    assert torch.cuda.is_available()
    return Plan()


def run(plan, A, B, ta, tb, pad_a=0, pad_b=0):
    """op(A) @ op(B) through the C ABI, operands stored with extra columns."""
    def stored(X, pad):
        S = torch.zeros(X.shape[0], X.shape[1] + pad, dtype=torch.float32, device="cuda")
        S[:, :X.shape[1]] = torch.from_numpy(X).cuda()
        return S[:, :X.shape[1]] if pad else S
    return gnn.dense_mm(stored(A, pad_a), stored(B, pad_b), plan, trans_a=ta, trans_b=tb)


def check(got, A, B, ta, tb):
    Ao = A.T if ta else A
    Bo = B.T if tb else B
    want = Ao.astype(np.float64) @ Bo.astype(np.float64)
    scale = np.abs(Ao).astype(np.float64) @ np.abs(Bo).astype(np.float64)
    K = Ao.shape[1]
    err = np.abs(got.cpu().numpy().astype(np.float64) - want)
    assert (err <= (K + 1) * U * scale + 1e-30).all(), float((err / np.maximum(scale, 1e-30)).max())


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (129, 257, 31), (300, 16, 256), (128, 128, 16),
                                   (77, 200, 1000), (5, 300, 17)])
@pytest.mark.parametrize("ta,tb", [(False, False), (False, True), (True, False), (True, True)])
def test_gemm_against_fp64(plan, M, N, K, ta, tb):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.normal(size=(K, M) if ta else (M, K)).astype(np.float32)
    B = rng.normal(size=(N, K) if tb else (K, N)).astype(np.float32)
    check(run(plan, A, B, ta, tb), A, B, ta, tb)
    # leading dimensions that are not multiples of 4 (scalar loads)
    check(run(plan, A, B, ta, tb, pad_a=1, pad_b=3), A, B, ta, tb)


def test_long_reduction_split_over_blocks(plan):
    """C^T * dY over many rows: the split reduction (fp64 partial sums)
    against fp64, and the same product without a workspace (one block per
    tile along K) gives values within the same bound."""
    rng = np.random.default_rng(5)
    n, d, dout = 70001, 130, 96
    Cd = rng.normal(size=(n, d)).astype(np.float32)
    dY = rng.normal(size=(n, dout)).astype(np.float32)
    nb = np.zeros(1, dtype=np.uint64)
    import ctypes
    b = ctypes.c_size_t()
    assert _lib.lib().spgemm_dense_gemm_workspace_bytes(plan.handle, d, dout, n, ctypes.byref(b)) == 0
    assert b.value >= 8 * d * dout                       # this reduction is split
    got = gnn.dense_mm(torch.from_numpy(Cd).cuda(), torch.from_numpy(dY).cuda(), plan,
                       trans_a=True)
    check(got, Cd, dY, True, False)
    # without a workspace
    Ct, Dt = torch.from_numpy(Cd).cuda(), torch.from_numpy(dY).cuda()
    out = torch.empty(d, dout, device="cuda")
    rc = _lib.lib().spgemm_dense_gemm(plan.handle, d, dout, n, ctypes.c_void_p(Ct.data_ptr()), d, 1,
                                      ctypes.c_void_p(Dt.data_ptr()), dout, 0,
                                      ctypes.c_void_p(out.data_ptr()), dout, None, 0, None)
    assert rc == _lib.OK
    torch.cuda.synchronize()
    check(out, Cd, dY, True, False)


def test_empty_and_invalid(plan):
    import ctypes
    L = _lib.lib()
    A = torch.zeros(4, 0, device="cuda")
    B = torch.zeros(0, 5, device="cuda")
    C = gnn.dense_mm(A, B, plan)
    assert C.shape == (4, 5) and bool((C == 0).all())
    out = torch.empty(4, 5, device="cuda")
    p = ctypes.c_void_p(out.data_ptr())
    assert L.spgemm_dense_gemm(plan.handle, -1, 5, 3, p, 3, 0, p, 5, 0, p, 5, None, 0, None) \
        == _lib.ERR_INVALID
    assert L.spgemm_dense_gemm(plan.handle, 4, 5, 3, p, 2, 0, p, 5, 0, p, 5, None, 0, None) \
        == _lib.ERR_INVALID                               # lda < K
    assert L.spgemm_dense_gemm(plan.handle, 4, 5, 3, p, 3, 2, p, 5, 0, p, 5, None, 0, None) \
        == _lib.ERR_INVALID                               # trans flag not 0/1
