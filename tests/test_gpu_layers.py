"""GPU parity of the pruned GNN layer (Section IV-C, Eqs. 1-3) against the
CPU oracle: TopK bit-exact, scatter/gather exact, the layer's forward and
backward within tolerances derived from the arithmetic:

  Y  = C * W with C from the SpGEMM (|C - C*| <= 1e-5 |A||T|) and an fp32
       GEMM over d terms: |Y - Y*| <= (1e-5 + gamma_d) |A||T||W|;
  dW = C^T * dY, an fp32 GEMM over n terms: (1e-5 + gamma_n) (|A||T|)^T |dY|;
  dX = M_k (.) A^T (dY W^T): an fp32 GEMM over dout terms, then the backward
       (fp64 sums, one fp32 rounding): (gamma_dout + 2u) |A|^T |dY| |W|^T,
with gamma_t = t * 2^-24 and u = 2^-24 (GEMMs in true fp32: TF32 off)."""
import numpy as np
import pytest
import torch

from oracle import layers
from paper_2512_12036_gb300 import DeviceCSR, Plan, gen
from paper_2512_12036_gb300 import gnn

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


@pytest.fixture(scope="module")
def plan():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.backends.cuda.matmul.allow_tf32 = False
    return Plan()


def dense_of(H: gen.HostCSR) -> np.ndarray:
    D = np.zeros((H.rows, H.cols))
    for i in range(H.rows):
        s, e = H.row_ptr[i], H.row_ptr[i + 1]
        np.add.at(D[i], H.col[s:e], H.val[s:e].astype(np.float64))
    return D


def features(n, d, seed, kind="normal"):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, d)).astype(np.float32)
    if kind == "ties":
        X = (np.round(X * 2) / 2).astype(np.float32)
    elif kind == "zeros":
        X[rng.random((n, d)) < 0.7] = 0.0
    elif kind == "special":
        specials = np.array([np.nan, np.inf, -np.inf, 0.0, -0.0], dtype=np.float32)
        m = rng.random((n, d)) < 0.2
        X[m] = rng.choice(specials, size=int(m.sum()))
        neg_nan = np.array([0xFFC00000, 0xFFFFFFFF], dtype=np.uint32).view(np.float32)
        X[0, :2] = neg_nan
    return X


@pytest.mark.parametrize("n,d,k,kind", [
    (1000, 256, 32, "normal"), (700, 256, 32, "ties"), (500, 256, 0, "normal"),
    (300, 256, 256, "normal"), (300, 100, 500, "zeros"), (257, 33, 7, "special"),
    (64, 2000, 100, "ties"), (40, 2000, 2000, "normal"), (1, 1, 1, "normal"), (0, 16, 4, "normal")])
def test_topk_bit_exact(plan, n, d, k, kind):
    X = features(n, d, seed=n + d + k, kind=kind)
    T = gnn.topk(torch.from_numpy(X).cuda(), k, plan)
    torch.cuda.synchronize()
    rp, col, val = layers.topk_csr(X, k)
    assert np.array_equal(T.row_ptr.cpu().numpy(), rp)
    assert np.array_equal(T.col.cpu().numpy(), col)
    assert np.array_equal(T.val.cpu().numpy().view(np.uint32), val.view(np.uint32))


def test_topk_strided_rows(plan):
    X = features(300, 80, seed=4)
    Xw = torch.zeros(300, 96, device="cuda")
    Xw[:, :80] = torch.from_numpy(X).cuda()
    T = gnn.topk(Xw[:, :80], 9, plan)
    rp, col, val = layers.topk_csr(X, 9)
    assert np.array_equal(T.col.cpu().numpy(), col)
    assert np.array_equal(T.val.cpu().numpy(), val)


def test_scatter_and_gather(plan):
    H = gen.random_csr(300, 90, 0.1, seed=6, duplicates=True)
    M = DeviceCSR.from_host(H)
    D = gnn.scatter_dense(M, plan)
    torch.cuda.synchronize()
    np.testing.assert_allclose(D.cpu().numpy(), dense_of(H), rtol=1e-6, atol=1e-6)
    R = torch.randn(300, 90, device="cuda")
    g = gnn.gather_dense(M, R, plan).cpu().numpy()
    Rh = R.cpu().numpy()
    rows = np.repeat(np.arange(300), np.diff(H.row_ptr))
    assert np.array_equal(g, Rh[rows, H.col])


def layer_problem(n=600, d=64, dout=32, k=8, seed=9):
    rng = np.random.default_rng(seed)
    Ah = gen.sym_normalised_adjacency(n, 12.0, rng)
    X = rng.normal(size=(n, d)).astype(np.float32)
    W = (rng.normal(size=(d, dout)) / np.sqrt(d)).astype(np.float32)
    dY = rng.normal(size=(n, dout)).astype(np.float32)
    return Ah, X, W, dY, k


def test_pruned_layer_forward_backward(plan):
    Ah, X, W, dY, k = layer_problem()
    n, d = X.shape
    dout = W.shape[1]
    A = DeviceCSR.from_host(Ah)
    Xt = torch.from_numpy(X).cuda().requires_grad_(True)
    Wt = torch.from_numpy(W).cuda().requires_grad_(True)
    Y = gnn.pruned_aggregation(A, Xt, Wt, k, plan)
    Y.backward(torch.from_numpy(dY).cuda())
    torch.cuda.synchronize()
    Ad = dense_of(Ah)
    Y64, _, _ = layers.layer_forward(Ad, X, W, k)
    dX64, dW64 = layers.layer_backward(Ad, X, W, k, dY)
    sY, sdX, sdW, _ = layers.layer_scales(Ad, X, W, k, dY)
    eY = np.abs(Y.detach().cpu().numpy() - Y64)
    assert (eY <= (1e-5 + d * U) * sY + 1e-30).all(), eY.max()
    edW = np.abs(Wt.grad.cpu().numpy() - dW64)
    assert (edW <= (1e-5 + n * U) * sdW + 1e-30).all(), edW.max()
    edX = np.abs(Xt.grad.cpu().numpy() - dX64)
    assert (edX <= (dout * U + 2 * U) * sdX + 1e-30).all(), edX.max()
    assert (Xt.grad.cpu().numpy()[~layers.topk_mask(X, k)] == 0).all()


def test_pruned_layer_no_pruning_equals_dense(plan):
    Ah, X, W, dY, _ = layer_problem(n=300, d=24, dout=16, seed=10)
    A = DeviceCSR.from_host(Ah)
    Y = gnn.pruned_aggregation(A, torch.from_numpy(X).cuda(), torch.from_numpy(W).cuda(),
                               X.shape[1], plan)
    Ad = dense_of(Ah)
    ref = Ad @ X.astype(np.float64) @ W.astype(np.float64)
    _, _, _, aC = layers.layer_scales(Ad, X, W, X.shape[1], dY)
    scale = aC @ np.abs(W.astype(np.float64))
    assert (np.abs(Y.cpu().numpy() - ref) <= (1e-5 + 24 * U) * scale + 1e-30).all()


def test_gcn_gin_sage_layers(plan):
    Ah, X, W, dY, k = layer_problem(n=400, d=48, dout=32, k=6, seed=11)
    A = DeviceCSR.from_host(Ah)
    Ad = dense_of(Ah)
    Xt = torch.from_numpy(X).cuda()
    # two-layer GCN, checked layer by layer (TopK of layer 2 sees the GPU's layer-1 output)
    gcn = gnn.PrunedGCN([48, 32, 16], k, plan)
    H1 = torch.relu(gnn.pruned_aggregation(A, Xt, gcn.W[0], k, plan)).detach()
    Y2 = gcn(A, Xt).detach().cpu().numpy()
    W2 = gcn.W[1].detach().cpu().numpy()
    H1h = H1.cpu().numpy()
    ref2, _, _ = layers.layer_forward(Ad, H1h, W2, k)
    s2, _, _, _ = layers.layer_scales(Ad, H1h, W2, k, np.zeros((400, 16)))
    assert (np.abs(Y2 - ref2) <= (1e-5 + 32 * U) * s2 + 1e-30).all()
    # GIN: relu((A + 2I) TopK(X) W1) W2, compared before the second linear map
    n = Ah.rows
    diag = np.arange(n)
    Ag = gen.csr_from_coo(n, n, np.concatenate([np.repeat(diag, np.diff(Ah.row_ptr)), diag]),
                          np.concatenate([Ah.col, diag]),
                          np.concatenate([Ah.val, np.full(n, 2.0, np.float32)]))
    gin = gnn.PrunedGIN(48, 32, 8, k, plan)
    W1 = gin.W1.detach().cpu().numpy()
    Hg = gnn.pruned_aggregation(DeviceCSR.from_host(Ag), Xt, gin.W1, k, plan).detach()
    refg, _, _ = layers.layer_forward(dense_of(Ag), X, W1, k)
    sg = layers.layer_scales(dense_of(Ag), X, W1, k, np.zeros((n, 32)))[0]
    assert (np.abs(Hg.cpu().numpy() - refg) <= (1e-5 + 48 * U) * sg + 1e-30).all()
    out_gin = gin(DeviceCSR.from_host(Ag), Xt)
    assert out_gin.shape == (n, 8) and torch.isfinite(out_gin).all()
    # GraphSAGE: TopK(X) Ws + mean_A TopK(X) Wn (the self term through the identity)
    deg = np.maximum(np.diff(Ah.row_ptr), 1).astype(np.float32)
    Am = gen.HostCSR(n, n, Ah.row_ptr, Ah.col,
                     (1.0 / np.repeat(deg, np.diff(Ah.row_ptr))).astype(np.float32))
    In = gen.csr_from_coo(n, n, diag, diag, np.ones(n, np.float32))
    sage = gnn.PrunedSAGE(48, 32, k, plan)
    Ys = sage(DeviceCSR.from_host(Am), DeviceCSR.from_host(In), Xt).detach().cpu().numpy()
    Ws = sage.Ws.detach().cpu().numpy()
    Wn = sage.Wn.detach().cpu().numpy()
    refs = (layers.layer_forward(np.eye(n), X, Ws, k)[0]
            + layers.layer_forward(dense_of(Am), X, Wn, k)[0])
    ss = (layers.layer_scales(np.eye(n), X, Ws, k, np.zeros((n, 32)))[0]
          + layers.layer_scales(dense_of(Am), X, Wn, k, np.zeros((n, 32)))[0])
    assert (np.abs(Ys - refs) <= (1e-5 + 48 * U + U) * ss + 1e-30).all()
