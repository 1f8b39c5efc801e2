"""Rows of many products on the GPU, against the CPU oracle.

* The 0.1 % fill workload of Section IV-B (random N x N matrices with round(0.001 N) entries per
  row): at N = 38000 every row of C gathers 38^2 = 1444 products, at N = 70000 4900: the block
  class B (its bit-vector form, B having at most 2^18 columns), and the dense class G when forced.  C is checked whole on the device (row pointer, strictly
  ascending columns in range) and 512 rows are compared with the oracle's product of those rows.
* The class-W orderings (the per-row "Combined" switch of Section IV-B): every forced ordering
  and the bit-vector threshold, on rows whose column ranges reach each ordering.
* Class G with many rows, spread over as many dense accumulators (CTAs) as the workspace holds.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1303_1651_gb300 import binding, synth
from tests.gpu_util import compare, gpu_product
from tests.sweep_util import check_structure, gpu_rows, sample_rows, sub_problem

pytestmark = pytest.mark.gpu

PATHS = pytest.mark.parametrize("fused", [False, True], ids=["3call", "fused"])


def device_product(A, B, opt=None):
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    ws = torch.empty(binding.spgemm_workspace_size(dA, dB, opt), dtype=torch.uint8, device="cuda")
    plan = binding.spgemm_plan(dA, dB, ws, opt)
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


@pytest.mark.parametrize("N,forced,cls", [(38_000, None, "B"), (38_000, "G", "G"), (70_000, None, "B"),
                                         (70_000, "G", "G")],
                         ids=["38000-block", "38000-dense", "70000-block", "70000-dense"])
def test_fill_one_per_mille(N, forced, cls):
    A = synth.random_fill(N, 0.001, synth.SEED_A + N)
    B = synth.random_fill(N, 0.001, synth.SEED_B + N)
    opt = binding.options(block_max_u=-1) if forced == "G" else None
    C_rp, C_col, C_val, nnz, info = device_product(A, B, opt)
    assert info["rows_per_class"][cls] == N, info["rows_per_class"]
    check_structure(C_rp, C_col, nnz, B.cols)
    rows = sample_rows(A.rows, seed=N)
    A_s, B_s = sub_problem(A, B, rows)
    compare(gpu_rows(C_rp, C_col, C_val, rows, B.cols), oracle.spgemm(A_s, B_s), single=True)


@PATHS
def test_many_dense_rows(fused):
    # about 700 rows of more than 4096 products: class G (the block class capped at 4096),
    # spread over the default number of slabs
    A = synth.random_lengths(np.full(700, 90), 3000, 461)
    B = synth.random_k(3000, 60, 462, ncols=20000)
    C = gpu_product(A, B, binding.options(block_max_u=4096), fused=fused)
    assert C["info"]["rows_per_class"]["G"] > 600, C["info"]["rows_per_class"]
    compare(C, oracle.spgemm(A, B))


@PATHS
@pytest.mark.parametrize("ncols,k,kb", [(20_000, 90, 60), (262_144, 60, 40), (262_145, 60, 40), (3_000_000, 45, 45),
                                        (1_000_000, 90, 80)],
                         ids=["one-window-5000", "one-window-limit", "two-windows", "many-windows",
                              "many-windows-7000"])
def test_block_class_windows(ncols, k, kb, fused):
    # class B orders a row by a bit vector over windows of 2^18 columns: one window when B has at
    # most 2^18 columns, else as many as the row's columns span (rows up to 8192 products)
    A = synth.random_lengths(np.full(500, k), 3000, 463)
    B = synth.random_k(3000, kb, 464, ncols=ncols)
    C = gpu_product(A, B, fused=fused)
    assert C["info"]["rows_per_class"]["B"] > 400, C["info"]["rows_per_class"]
    compare(C, oracle.spgemm(A, B), single=True)


ORDERINGS = [dict(warp_order=1), dict(warp_order=2), dict(warp_order=3), dict(warp_bitvec_ratio=2),
             dict(warp_bitvec_ratio=32), dict()]


@pytest.mark.parametrize("order", ORDERINGS, ids=["bitvec", "regsort", "hash", "ratio2", "ratio32", "auto"])
@PATHS
def test_warp_orderings(order, fused):
    # rows of 9..32 entries of A times rows of 9..20 entries of B (class W: 81..640 products);
    # B's column count sets each row's column range, so one matrix reaches every ordering
    for ncols, seed in ((1500, 471), (200_000, 472), (20_000_000, 473)):
        A = synth.random_lengths(np.random.default_rng(seed).integers(9, 33, 600), 500, seed)
        B = synth.random_lengths(np.random.default_rng(seed + 1).integers(9, 21, 500), ncols, seed + 1)
        C = gpu_product(A, B, binding.options(m1_max_u=-1, m2_max_u=-1, warp_max_u=1024, **order), fused=fused)
        assert C["info"]["rows_per_class"]["W"] > 500
        compare(C, oracle.spgemm(A, B), single=True)
