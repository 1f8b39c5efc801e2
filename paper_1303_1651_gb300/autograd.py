"""torch.autograd.Function for C = A*B on fixed CSR structures, differentiable in the values.

Forward: plan + single-pass compute (C's structure from the structures of A and B).
Backward: dA = (dC B^T) restricted to A's structure, dB = (A^T dC) restricted to B's structure,
computed by the library's sampled-product kernels (spgemm_backward).  Only the value arrays are
differentiable; the structures are constants.
"""
from __future__ import annotations

import torch

from . import binding


class _PlanHolder:
    """Owns a plan for the lifetime of an autograd context (backward may run more than once)."""

    def __init__(self, plan):
        self.plan = plan

    def __del__(self):
        try:
            binding.spgemm_free(self.plan)
        except Exception:
            pass


class SpGEMMFunction(torch.autograd.Function):
    """C_val = SpGEMMFunction.apply(A_val, B_val, A_struct, B_struct).

    A_struct, B_struct: binding.DeviceCSR whose row_ptr/col_idx give the structures (their val
    tensors are ignored).  Returns C's values; C's structure is attached to the returned tensor's
    context and available as SpGEMMFunction.last_structure (row_ptr, col_idx, shape).
    """

    last_structure = None

    @staticmethod
    def forward(ctx, A_val, B_val, A_struct: binding.DeviceCSR, B_struct: binding.DeviceCSR):
        A = binding.DeviceCSR(A_struct.rows, A_struct.cols, A_struct.row_ptr, A_struct.col_idx, A_val.detach())
        B = binding.DeviceCSR(B_struct.rows, B_struct.cols, B_struct.row_ptr, B_struct.col_idx, B_val.detach())
        dev = A.row_ptr.device
        ws = torch.empty(binding.spgemm_workspace_size(A, B), dtype=torch.uint8, device=dev)
        plan = binding.spgemm_plan(A, B, ws)
        F = binding.spgemm_plan_info(plan)["products"]
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
        C_col = torch.empty(max(F, 1), dtype=torch.int32, device=dev)
        C_val = torch.empty(max(F, 1), dtype=A_val.dtype, device=dev)
        nnz = binding.spgemm_compute(plan, A.val, B.val, C_rp, C_col, C_val)
        C_col, C_val = C_col[:nnz], C_val[:nnz]
        ctx.holder = _PlanHolder(plan)
        ctx.ws = ws
        ctx.A, ctx.B = A, B
        ctx.C = (C_rp, C_col)
        ctx.save_for_backward(A_val, B_val)
        SpGEMMFunction.last_structure = (C_rp, C_col, (A.rows, B.cols))
        return C_val

    @staticmethod
    def backward(ctx, dC):
        A_val, B_val = ctx.saved_tensors
        dC = dC.contiguous().to(torch.float64)
        dA = torch.empty_like(A_val) if ctx.needs_input_grad[0] else None
        dB = torch.empty_like(B_val) if ctx.needs_input_grad[1] else None
        tws = None
        if dB is not None:
            tws = torch.empty(binding.spgemm_backward_workspace_size(ctx.A, ctx.B), dtype=torch.uint8,
                              device=A_val.device)
        # the plan still refers to C's structure tensors kept in ctx.C
        plan = ctx.holder.plan
        binding.spgemm_backward(plan, A_val.detach(), B_val.detach(), dC, dA, dB, tws)
        binding.spgemm_status(plan)
        return dA, dB, None, None


def spgemm(A_val, B_val, A_struct, B_struct):
    """Differentiable C_val for C = A*B (see SpGEMMFunction)."""
    return SpGEMMFunction.apply(A_val, B_val, A_struct, B_struct)
