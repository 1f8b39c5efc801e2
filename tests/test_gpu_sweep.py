"""The size sweep: 13 log-spaced N = round(10^(3 + i/3)) from 1e3 to 1e7, for the Laplacian²
(grid side round(sqrt(N))) and for random·random with 4, 8 and 16 distinct columns per row, through
the single-pass product (plan, then compute with C sized by F): the path the sweep bench times.

Up to N = 1e5 every entry is compared with the oracle.  Above, C stays on the device and is checked
whole against what holds at any size: the row pointer runs from 0 to nnz(C) without decreasing,
columns ascend strictly within every row and lie in [0, n), nnz(C) <= F, and F equals the count of
products (the lengths of the rows of B summed over the entries of A).  The Laplacian² is compared
entry by entry with its closed form (13 entries on interior rows: 20 on the diagonal, -8 at grid
distance 1, 2 on the grid diagonals, 1 at distance 2; the diagonal is 16 + the number of grid
neighbours).  For random·random, 512 rows (the first, the last and a seeded sample) are compared
with the oracle's product of those rows of A with the rows of B they reference.

At N = 1e7 with 16 per row, nnz(C) passes INT32_MAX: both paths must report the overflow without
writing outside their buffers."""
import numpy as np
import pytest
import torch

import oracle
from paper_1303_1651_gb300 import synth
from tests.gpu_util import compare
from tests.sweep_util import check_structure, gpu_rows, laplacian_square, products_count, sample_rows, sub_problem

pytestmark = pytest.mark.gpu

FULL_LIMIT = 100_000          # sizes up to this are compared with the oracle entry by entry
OVERFLOW_POINT = (10_000_000, "rand16")
POINTS = [p for p in synth.sweep_points() if p != OVERFLOW_POINT]


def device_product(A, B):
    """plan -> C sized by F -> spgemm_compute; C stays on the device."""
    from paper_1303_1651_gb300 import binding
    dA = binding.DeviceCSR.from_host(A)
    dB = dA if B is A else binding.DeviceCSR.from_host(B)
    ws = torch.empty(binding.spgemm_workspace_size(dA, dB), dtype=torch.uint8, device="cuda")
    plan = binding.spgemm_plan(dA, dB, ws)
    try:
        info = binding.spgemm_plan_info(plan)
        F = info["products"]
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device="cuda")
        C_col = torch.empty(max(F, 1), dtype=torch.int32, device="cuda")
        C_val = torch.empty(max(F, 1), dtype=torch.float64, device="cuda")
        nnz = binding.spgemm_compute(plan, dA.val, dB.val, C_rp, C_col, C_val)
    finally:
        binding.spgemm_free(plan)
    torch.cuda.synchronize()
    return C_rp, C_col[:nnz], C_val[:nnz], nnz, info


@pytest.mark.parametrize("N,kind", POINTS, ids=[f"N{N}-{k}" for N, k in POINTS])
def test_sweep_point(N, kind):
    A, B = synth.sweep_problem(N, kind)
    C_rp, C_col, C_val, nnz, info = device_product(A, B)
    F = products_count(A, B)
    assert info["products"] == F
    assert nnz <= F
    check_structure(C_rp, C_col, nnz, B.cols)
    if kind == "lap":
        n = int(round(np.sqrt(A.rows)))
        assert nnz == 13 * n * n - 20 * n + 4 and F == 25 * (n - 2) ** 2 + 64 * (n - 2) + 36
        rp, col, val = laplacian_square(n)
        assert torch.equal(C_rp.long(), rp) and torch.equal(C_col.long(), col) and torch.equal(C_val, val)
    if N <= FULL_LIMIT:
        out = dict(rows=A.rows, cols=B.cols, row_ptr=C_rp.cpu().numpy(), col_idx=C_col.cpu().numpy(),
                   val=C_val.cpu().numpy())
        compare(out, oracle.spgemm(A, B), exact=kind == "lap", single=True)
    elif kind != "lap":
        rows = sample_rows(A.rows, seed=N)
        A_sub, B_sub = sub_problem(A, B, rows)
        compare(gpu_rows(C_rp, C_col, C_val, rows, B.cols), oracle.spgemm(A_sub, B_sub), single=True)


def test_sweep_overflow_point():
    """N = 1e7, 16 per row: F = 2.56e9 products and nnz(C) beyond INT32_MAX."""
    from paper_1303_1651_gb300 import binding
    A, B = synth.sweep_problem(*OVERFLOW_POINT)
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    del A, B
    ws = torch.empty(binding.spgemm_workspace_size(dA, dB), dtype=torch.uint8, device="cuda")
    C_rp = torch.empty(dA.rows + 1, dtype=torch.int32, device="cuda")
    # three calls: the symbolic pass reports the overflow and leaves no structure behind
    plan = binding.spgemm_plan(dA, dB, ws)
    try:
        assert binding.spgemm_plan_info(plan)["products"] == 16 * 16 * 10_000_000
        with pytest.raises(binding.SpgemmError) as e:
            binding.spgemm_symbolic(plan, C_rp)
        assert e.value.name == "SPGEMM_ERR_OVERFLOW"
        rp = C_rp.long()
        assert int(rp[0]) == 0 and bool((rp[1:] >= rp[:-1]).all()) and int(rp[-1]) == (1 << 31) - 1
        dummy = torch.empty(1, dtype=torch.int32, device="cuda")
        with pytest.raises(binding.SpgemmError) as e:
            binding.spgemm_numeric(plan, dA.val, dB.val, dummy, dummy.double())
        assert e.value.name == "SPGEMM_ERR_STATE"
    finally:
        binding.spgemm_free(plan)
    # single pass with a small capacity: the overflow, nothing written past the capacity
    plan = binding.spgemm_plan(dA, dB, ws)
    try:
        cap = 1 << 20
        C_col = torch.full((cap + 4096,), -7, dtype=torch.int32, device="cuda")
        C_val = torch.full((cap + 4096,), 5.0, dtype=torch.float64, device="cuda")
        with pytest.raises(binding.SpgemmError) as e:
            binding.spgemm_compute(plan, dA.val, dB.val, C_rp, C_col[:cap], C_val[:cap])
        assert e.value.name == "SPGEMM_ERR_OVERFLOW"
        assert bool((C_col[cap:] == -7).all()) and bool((C_val[cap:] == 5.0).all())
        rp = C_rp.long()
        assert int(rp.min()) >= 0 and int(rp.max()) <= cap and bool((rp[1:] >= rp[:-1]).all())
    finally:
        binding.spgemm_free(plan)
