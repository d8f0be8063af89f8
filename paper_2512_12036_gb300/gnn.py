"""GNN layers with a pruning (top-k) layer on the SpGEMM (Section IV-C).

Eq. 1: X_l = A * TopK(X_{l-1}, k) * W_l. The forward takes TopK of the
dense features into CSR (the mask M_k of Eq. 2 and its values), multiplies
A by it with the hash-based SpGEMM, and applies the dense weight. The
backward follows Eq. 3: the gradient of A * TopK(X) is dY * W^T read at that
product's pattern, spgemm_backward turns it into A^T * dC on TopK's pattern
(the M_k-masked gradient of Eq. 3), and a scatter lays it into the dense
dX. The products with the dense W (C*W, dY*W^T, C^T*dY) are this library's
fp32 GEMM (spgemm_dense_gemm); every step of the layer runs in its kernels.

GCN, GIN and GraphSAGE layers are compositions of that step (the graph
operator each uses is built by the caller: Ahat = D^-1/2 (A+I) D^-1/2 for
GCN, A + (1+eps) I for GIN, the row-normalised A for GraphSAGE's mean).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import check
from .api import DeviceCSR, Plan, _ptr, _stream


def _small_ws(plan: Plan, device) -> torch.Tensor:
    """An initialised 1 KB workspace (status word) for the scatter and gather."""
    ws = torch.empty(1024 + 256, dtype=torch.uint8, device=device)
    off = (-ws.data_ptr()) % 256
    ws = ws[off:off + 1024]
    plan.workspace_init(ws)
    return ws


def topk(X: torch.Tensor, k: int, plan: Plan, stream=None) -> DeviceCSR:
    """TopK(X, k) of Eq. 2 for a dense row-major fp32 matrix: CSR with
    min(k, d) entries per row in column order."""
    if X.dtype != torch.float32 or X.dim() != 2 or (X.numel() > 0 and X.stride(1) != 1):
        raise ValueError("X must be a 2-D fp32 tensor with unit column stride")
    n, d = X.shape
    kk = max(0, min(k, d))
    ldx = X.stride(0) if X.numel() > 0 else d
    rp = torch.empty(n + 1, dtype=torch.int32, device=X.device)
    col = torch.empty(n * kk, dtype=torch.int32, device=X.device)
    val = torch.empty(n * kk, dtype=torch.float32, device=X.device)
    check(_lib.lib().spgemm_topk_dense(plan.handle, _ptr(X), n, d, ldx, k, _ptr(rp),
                                       _ptr(col), _ptr(val), _stream(stream)),
          "spgemm_topk_dense")
    return DeviceCSR(n, d, rp, col, val)


def scatter_dense(M: DeviceCSR, plan: Plan, vals: torch.Tensor | None = None,
                  out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """out += M as a dense matrix (values ``vals`` on M's pattern if given)."""
    if out is None:
        out = torch.zeros(M.rows, M.cols, dtype=torch.float32, device=M.device)
    if ws is None:
        ws = _small_ws(plan, M.device)
    v = _ptr(vals) if vals is not None else None
    check(_lib.lib().spgemm_csr_scatter_dense(plan.handle, ctypes.byref(M.struct()), v, _ptr(out),
                                              out.stride(0), _ptr(ws), ws.numel(),
                                              _stream(stream)),
          "spgemm_csr_scatter_dense")
    return out


def gather_dense(M: DeviceCSR, D: torch.Tensor, plan: Plan, ws: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """Values of the dense matrix D at M's pattern."""
    out = torch.empty(M.nnz, dtype=torch.float32, device=M.device)
    if ws is None:
        ws = _small_ws(plan, M.device)
    check(_lib.lib().spgemm_csr_gather_dense(plan.handle, ctypes.byref(M.struct()), _ptr(D),
                                             D.stride(0), _ptr(out), _ptr(ws), ws.numel(),
                                             _stream(stream)),
          "spgemm_csr_gather_dense")
    return out


def dense_mm(A: torch.Tensor, B: torch.Tensor, plan: Plan, trans_a: bool = False,
             trans_b: bool = False, stream=None) -> torch.Tensor:
    """op(A) @ op(B) for row-major fp32 device matrices with unit column
    stride, through spgemm_dense_gemm (a split-K workspace is allocated when
    the reduction is long)."""
    for T in (A, B):
        if T.dtype != torch.float32 or T.dim() != 2 or (T.numel() > 0 and T.stride(1) != 1):
            raise ValueError("operands must be 2-D fp32 tensors with unit column stride")
    M, K = (A.shape[1], A.shape[0]) if trans_a else (A.shape[0], A.shape[1])
    Kb, N = (B.shape[1], B.shape[0]) if trans_b else (B.shape[0], B.shape[1])
    if K != Kb:
        raise ValueError(f"inner dimensions differ: {K} vs {Kb}")
    C = torch.empty(M, N, dtype=torch.float32, device=A.device)
    L = _lib.lib()
    nb = ctypes.c_size_t()
    check(L.spgemm_dense_gemm_workspace_bytes(plan.handle, M, N, K, ctypes.byref(nb)),
          "spgemm_dense_gemm_workspace_bytes")
    ws = None
    if nb.value:
        raw = torch.empty(int(nb.value) + 256, dtype=torch.uint8, device=A.device)
        off = (-raw.data_ptr()) % 256
        ws = raw[off:off + int(nb.value)]
    lda = A.stride(0) if A.numel() else A.shape[1]
    ldb = B.stride(0) if B.numel() else B.shape[1]
    check(L.spgemm_dense_gemm(plan.handle, M, N, K, _ptr(A), lda, int(trans_a), _ptr(B), ldb,
                              int(trans_b), _ptr(C), N, _ptr(ws) if ws is not None else None,
                              int(nb.value) if ws is not None else 0, _stream(stream)),
          "spgemm_dense_gemm")
    return C


class DenseLinear(torch.autograd.Function):
    """Y = X @ W with both gradients (dX = dY W^T, dW = X^T dY) through
    spgemm_dense_gemm."""

    @staticmethod
    def forward(ctx, X, W, plan: Plan):
        X = X.detach().contiguous()
        W = W.detach().contiguous()
        ctx.save_for_backward(X, W)
        ctx.plan = plan
        return dense_mm(X, W, plan)

    @staticmethod
    def backward(ctx, dY):
        X, W = ctx.saved_tensors
        dY = dY.contiguous()
        dX = dense_mm(dY, W, ctx.plan, trans_b=True) if ctx.needs_input_grad[0] else None
        dW = dense_mm(X, dY, ctx.plan, trans_a=True) if ctx.needs_input_grad[1] else None
        return dX, dW, None


def dense_linear(X: torch.Tensor, W: torch.Tensor, plan: Plan) -> torch.Tensor:
    return DenseLinear.apply(X, W, plan)


class PrunedAggregation(torch.autograd.Function):
    """Y = A * TopK(X, k) * W (Eq. 1) with the backward of Eq. 3."""

    @staticmethod
    def forward(ctx, X, W, A: DeviceCSR, k: int, plan: Plan):
        X = X.detach().contiguous()
        W = W.detach().contiguous()
        ws = _small_ws(plan, X.device)
        T = topk(X, k, plan)
        C = plan.spgemm(A, T)
        Cd = scatter_dense(C, plan, ws=ws)
        plan.check_status(ws, "pruned layer forward")
        ctx.save_for_backward(Cd, W)
        ctx.A, ctx.T, ctx.C, ctx.plan, ctx.shape = A, T, C, plan, X.shape
        return dense_mm(Cd, W, plan)

    @staticmethod
    def backward(ctx, dY):
        Cd, W = ctx.saved_tensors
        plan = ctx.plan
        dY = dY.contiguous()
        dX = dW = None
        if ctx.needs_input_grad[1]:
            dW = dense_mm(Cd, dY, plan, trans_a=True)
        if ctx.needs_input_grad[0]:
            ws = _small_ws(plan, dY.device)
            dC = gather_dense(ctx.C, dense_mm(dY, W, plan, trans_b=True), plan, ws=ws)
            bws = plan.backward_workspace(ctx.A, ctx.T)
            _, dT = plan.backward(ctx.A, ctx.T, ctx.C, dC, need_dA=False, need_dB=True, ws=bws)
            plan.check_status(bws, "pruned layer backward")
            dX = scatter_dense(ctx.T, plan, vals=dT, ws=ws)
            plan.check_status(ws, "pruned layer backward")
        return dX, dW, None, None, None


def pruned_aggregation(A: DeviceCSR, X: torch.Tensor, W: torch.Tensor, k: int,
                       plan: Plan | None = None) -> torch.Tensor:
    """Eq. 1: A * TopK(X, k) * W, differentiable in X and W."""
    plan = plan or Plan(device=X.device.index)
    return PrunedAggregation.apply(X, W, A, k, plan)


class PrunedGCN(torch.nn.Module):
    """Stacked GCN layers X_l = act(Ahat * TopK(X_{l-1}, k) * W_l)."""

    def __init__(self, dims: list[int], k: int, plan: Plan | None = None, device="cuda"):
        super().__init__()
        g = torch.Generator().manual_seed(0)
        self.W = torch.nn.ParameterList([
            torch.nn.Parameter((torch.randn(a, b, generator=g) / a ** 0.5).to(device))
            for a, b in zip(dims, dims[1:])])
        self.k = k
        self.plan = plan or Plan(device=torch.device(device).index)

    def forward(self, Ahat: DeviceCSR, X: torch.Tensor) -> torch.Tensor:
        for q, W in enumerate(self.W):
            X = pruned_aggregation(Ahat, X, W, self.k, self.plan)
            if q + 1 < len(self.W):
                X = torch.relu(X)
        return X


class PrunedGIN(torch.nn.Module):
    """GIN layer with pruning: MLP((A + (1+eps) I) * TopK(X, k)); the first
    linear map of the MLP is fused into the pruned aggregation."""

    def __init__(self, d_in: int, d_hidden: int, d_out: int, k: int, plan: Plan | None = None,
                 device="cuda"):
        super().__init__()
        g = torch.Generator().manual_seed(1)
        self.W1 = torch.nn.Parameter((torch.randn(d_in, d_hidden, generator=g) / d_in ** 0.5).to(device))
        self.W2 = torch.nn.Parameter((torch.randn(d_hidden, d_out, generator=g) / d_hidden ** 0.5).to(device))
        self.k = k
        self.plan = plan or Plan(device=torch.device(device).index)

    def forward(self, A_gin: DeviceCSR, X: torch.Tensor) -> torch.Tensor:
        return dense_linear(torch.relu(pruned_aggregation(A_gin, X, self.W1, self.k, self.plan)),
                            self.W2, self.plan)


class PrunedSAGE(torch.nn.Module):
    """GraphSAGE layer with pruning: TopK(X) * W_self + mean_A * TopK(X) * W_neigh.
    The self term is the pruned aggregation with the identity operator."""

    def __init__(self, d_in: int, d_out: int, k: int, plan: Plan | None = None, device="cuda"):
        super().__init__()
        g = torch.Generator().manual_seed(2)
        self.Ws = torch.nn.Parameter((torch.randn(d_in, d_out, generator=g) / d_in ** 0.5).to(device))
        self.Wn = torch.nn.Parameter((torch.randn(d_in, d_out, generator=g) / d_in ** 0.5).to(device))
        self.k = k
        self.plan = plan or Plan(device=torch.device(device).index)

    def forward(self, A_mean: DeviceCSR, I_n: DeviceCSR, X: torch.Tensor) -> torch.Tensor:
        return (pruned_aggregation(I_n, X, self.Ws, self.k, self.plan)
                + pruned_aggregation(A_mean, X, self.Wn, self.k, self.plan))
