"""torch.autograd.Function over the SpGEMM forward and its hand-written backward.

For the pruned-GNN aggregation C = A_hat * X (Eq. 1-3): the forward is the
hash-based multi-phase product; the backward calls spgemm_backward, which
returns dA_vals (an SDDMM of dC * X^T at A_hat's pattern) and dX_vals
(A_hat^T * dC at X's pattern, i.e. the gradient masked by X's top-k pattern
M_k, as Eq. 3 states). Structures are fixed; only stored values carry grads.
"""
from __future__ import annotations

import torch

from .api import DeviceCSR, Plan


class SpGEMMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a_vals, b_vals, A: DeviceCSR, B: DeviceCSR, plan: Plan):
        Av = DeviceCSR(A.rows, A.cols, A.row_ptr, A.col, a_vals.detach().contiguous())
        Bv = DeviceCSR(B.rows, B.cols, B.row_ptr, B.col, b_vals.detach().contiguous())
        C = plan.spgemm(Av, Bv)
        ctx.plan = plan
        ctx.A, ctx.B, ctx.C = Av, Bv, C
        ctx.mark_non_differentiable(C.row_ptr, C.col)
        return C.row_ptr, C.col, C.val

    @staticmethod
    def backward(ctx, g_rowptr, g_col, g_val):
        need_a, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if g_val is None or not (need_a or need_b):
            return None, None, None, None, None
        ws = ctx.plan.backward_workspace(ctx.A, ctx.B)
        dA, dB = ctx.plan.backward(ctx.A, ctx.B, ctx.C, g_val, need_dA=need_a, need_dB=need_b,
                                   ws=ws)
        ctx.plan.check_status(ws, "spgemm_backward")
        return dA, dB, None, None, None


def spgemm(a_vals: torch.Tensor, b_vals: torch.Tensor, A: DeviceCSR, B: DeviceCSR,
           plan: Plan | None = None) -> DeviceCSR:
    """C = A*B with gradients flowing to ``a_vals`` and ``b_vals`` (the stored
    values of A and B; A and B provide the structure)."""
    plan = plan or Plan(device=A.device.index)
    rp, col, val = SpGEMMFunction.apply(a_vals, b_vals, A, B, plan)
    return DeviceCSR(A.rows, B.cols, rp, col, val)
