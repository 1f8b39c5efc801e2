"""Shared helpers for the GPU parity tests: run the CUDA path, compare with the oracle."""
from __future__ import annotations

import numpy as np

import oracle

TOL = 1e-12   # |c - c_ref| / sum |a*b| per entry (max relative error of the product in FP64)


def gpu_product(A, B, opt=None, stream=None, fused=False):
    """C = A*B through the C ABI: plan/symbolic/numeric, or plan/compute (fused=True)."""
    import torch
    from paper_1303_1651_gb300 import binding
    dA = binding.DeviceCSR.from_host(A)
    dB = dA if B is A else binding.DeviceCSR.from_host(B)
    if not fused:
        prod = binding.Product(dA, dB, opt, stream)
        try:
            C = prod.numeric(stream=stream)
            binding.spgemm_status(prod.plan, stream)
            torch.cuda.synchronize()
            out = C.to_host()
            out["info"] = prod.info
            return out
        finally:
            prod.close()
    ws = torch.empty(binding.spgemm_workspace_size(dA, dB, opt), dtype=torch.uint8, device="cuda")
    plan = binding.spgemm_plan(dA, dB, ws, opt, stream)
    try:
        info = binding.spgemm_plan_info(plan)
        F = info["products"]
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device="cuda")
        C_col = torch.full((max(F, 1),), -7, dtype=torch.int32, device="cuda")
        C_val = torch.full((max(F, 1),), float("nan"), dtype=torch.float64, device="cuda")
        nnz = binding.spgemm_compute(plan, dA.val, dB.val, C_rp, C_col, C_val, stream)
        torch.cuda.synchronize()
        out = dict(rows=A.rows, cols=B.cols, row_ptr=C_rp.cpu().numpy(), col_idx=C_col[:nnz].cpu().numpy(),
                   val=C_val[:nnz].cpu().numpy(), nnz=nnz, info=info)
        # nothing written past nnz(C)
        assert bool((C_col[nnz:] == -7).all()), "fused pass wrote beyond nnz(C)"
        return out
    finally:
        binding.spgemm_free(plan)


def compare(C: dict, R: dict, tol: float = TOL, exact: bool = False, single: bool = False) -> dict:
    """Pattern bit-exact; values within tol of sum|a*b|.  exact=True: every value bit-exact (inputs
    whose sums are exact, e.g. small integers).  single=True: entries made of one product bit-exact
    (a*b rounded once on both sides)."""
    rp = np.asarray(C["row_ptr"], np.int64)
    assert rp.shape == R["row_ptr"].shape, "row_ptr length"
    assert np.array_equal(rp, R["row_ptr"]), f"row_ptr differs at {np.nonzero(rp != R['row_ptr'])[0][:5]}"
    col = np.asarray(C["col_idx"], np.int64)
    assert np.array_equal(col, R["col_idx"]), f"col_idx differs at {np.nonzero(col != R['col_idx'])[0][:5]}"
    v, rv, ab = np.asarray(C["val"]), R["val"], R["absval"]
    diff = np.abs(v - rv)
    scale = np.where(ab > 0, ab, 1.0)
    err = diff / scale
    maxerr = float(err.max()) if err.size else 0.0
    nz = rv != 0
    plain = float((diff[nz] / np.abs(rv[nz])).max()) if nz.any() else 0.0
    if exact:
        assert np.array_equal(v, rv), f"values differ (max scaled err {maxerr:.3e})"
    if single:
        one = R["count"] == 1
        assert np.array_equal(v[one], rv[one]), "single-product entries differ"
    assert maxerr <= tol, f"max |c-c_ref|/sum|ab| = {maxerr:.3e} > {tol}"
    return dict(max_err=maxerr, max_plain_rel=plain, nnz=int(rp[-1]))
