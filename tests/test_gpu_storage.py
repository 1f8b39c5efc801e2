"""Operands in compressed columns (CSC) and the torch front door, against the CPU oracle.

Section IV-A of the paper multiplies matrices stored in different orders by converting one of
them first.  Here a CSC operand is converted inside the library (plan: its structure, by the
counting-sort transpose; each call: its values, gathered through the recorded permutation), so
the product must equal the oracle's product of the same matrix in compressed rows, element by
element: pattern bit-exact, values within 1e-12 of sum |a*b|, single-product entries bit-exact.
The CSC inputs are built on the host by the oracle's transpose (pinned to the dense transpose)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1303_1651_gb300 import binding, synth
from tests.gpu_util import compare

pytestmark = pytest.mark.gpu

PATHS = pytest.mark.parametrize("fused", [False, True], ids=["3call", "fused"])
LAYOUTS = pytest.mark.parametrize("layout", ["csr-csc", "csc-csr", "csc-csc"])


def dev_csc(M):
    """Host CSR -> device CSC (column pointers, row indices ascending in each column, values)."""
    cp, ri, v = oracle.transpose(M)
    return binding.DeviceCSC(M.rows, M.cols, torch.from_numpy(cp.astype(np.int32)).cuda(),
                             torch.from_numpy(ri.astype(np.int32)).cuda(), torch.from_numpy(v).cuda())


def operands(A, B, layout):
    a = dev_csc(A) if layout.startswith("csc") else binding.DeviceCSR.from_host(A)
    b = dev_csc(B) if layout.endswith("csc") else binding.DeviceCSR.from_host(B)
    return a, b


def run(a, b, fused, opt=None):
    if fused:
        C = binding.multiply_fused(a, b, opt)
    else:
        C = binding.multiply(a, b, opt, check=True)
    torch.cuda.synchronize()
    return C.to_host()


@LAYOUTS
@PATHS
def test_random_rectangular(layout, fused):
    A = synth.random_k(1700, 5, 401, ncols=1300)
    B = synth.random_k(1300, 6, 402, ncols=900)
    a, b = operands(A, B, layout)
    compare(run(a, b, fused), oracle.spgemm(A, B), single=True)


@LAYOUTS
@PATHS
def test_laplacian_exact(layout, fused):
    L = synth.laplacian5(40)
    a, b = operands(L, L, layout)
    compare(run(a, b, fused), oracle.spgemm(L, L), exact=True)


@PATHS
def test_every_class_with_csc_b(fused):
    # rows of every class: the conversion feeds the sort, warp, block and dense kernels alike
    A = synth.power_law(2000, 1500, 3, alpha=1.5, max_len=1500)
    B = synth.power_law(1500, 2500, 4, alpha=1.5, max_len=300)
    a, b = operands(A, B, "csr-csc")
    C = binding.Product(a, b)
    try:
        got = C.numeric().to_host()
        binding.spgemm_status(C.plan)
        cls = C.info["rows_per_class"]
    finally:
        C.close()
    compare(got, oracle.spgemm(A, B))
    assert all(cls[c] > 0 for c in ("M1", "M2", "W", "B", "G")), cls


def test_unsorted_and_repeated_rows_in_a_column():
    # A CSC column may list its rows in any order and repeat one.  The converted row keeps the
    # entries by column, then by their position in the given arrays: the equivalent compressed
    # rows are the entries sorted stably by (row, column).
    rng = np.random.default_rng(7)
    rows, cols, nnz = 300, 250, 2400
    r = rng.integers(0, rows, nnz)
    c = np.sort(rng.integers(0, cols, nnz))
    v = rng.uniform(-1, 1, nnz)
    r[5:9] = r[4]                                  # repeats within column c[4]
    c[5:9] = c[4]
    order = rng.permutation(nnz)                   # shuffle rows within each column, keep column order
    order = order[np.argsort(c[order], kind="stable")]
    r, c, v = r[order], c[order], v[order]
    cp = np.zeros(cols + 1, np.int64)
    np.add.at(cp, c + 1, 1)
    cp = np.cumsum(cp)
    a = binding.DeviceCSC(rows, cols, torch.from_numpy(cp.astype(np.int32)).cuda(),
                          torch.from_numpy(r.astype(np.int32)).cuda(), torch.from_numpy(v).cuda())
    srt = np.lexsort((c, r))                       # stable: equal (row, column) keep their order
    Acsr = synth.CSR(rows, cols, np.concatenate([[0], np.cumsum(np.bincount(r, minlength=rows))]).astype(np.int32),
                     c[srt].astype(np.int32), v[srt])
    B = synth.random_k(cols, 7, 409, ncols=333)
    b = binding.DeviceCSR.from_host(B)
    for fused in (False, True):
        compare(run(a, b, fused), oracle.spgemm(Acsr, B))


def test_numeric_again_with_new_csc_values():
    A = synth.random_k(2500, 4, 411, ncols=2000)
    B = synth.random_k(2000, 7, 412, ncols=2100)
    a, b = operands(A, B, "csc-csc")
    prod = binding.Product(a, b)
    try:
        compare(prod.numeric().to_host(), oracle.spgemm(A, B), single=True)
        A2, B2 = A.copy(), B.copy()
        A2.val = np.cos(3.0 * A.val)
        B2.val = -0.5 * B.val + 0.25
        a2v = torch.from_numpy(oracle.transpose(A2)[2]).cuda()
        b2v = torch.from_numpy(oracle.transpose(B2)[2]).cuda()
        got = prod.numeric(a2v, b2v).to_host()
        binding.spgemm_status(prod.plan)
        compare(got, oracle.spgemm(A2, B2), single=True)
        # pattern reuse on the converted structure gives the same values again
        C = prod.numeric(a2v, b2v)
        prod.record(C)
        rep = prod.replay(a2v, b2v).to_host()
        binding.spgemm_status(prod.plan)
        compare(rep, oracle.spgemm(A2, B2), single=True)
    finally:
        prod.close()


def to_csc_order(M, vals):
    """Values aligned with M's CSR entries, reordered as M's CSC entries."""
    T = M.copy()
    T.val = np.asarray(vals, np.float64)
    return oracle.transpose(T)[2]


@LAYOUTS
def test_backward_returns_gradients_in_the_given_order(layout):
    A = synth.random_k(1200, 6, 421, ncols=900)
    B = synth.random_k(900, 5, 422, ncols=1000)
    a, b = operands(A, B, layout)
    opt = binding.with_storage(a, b)
    ws = torch.empty(binding.spgemm_workspace_size(a, b, opt), dtype=torch.uint8, device="cuda")
    tws = torch.empty(binding.spgemm_backward_workspace_size(binding.DeviceCSR.from_host(A),
                                                             binding.DeviceCSR.from_host(B)),
                      dtype=torch.uint8, device="cuda")
    plan = binding.spgemm_plan(a, b, ws, opt)
    try:
        F = binding.spgemm_plan_info(plan)["products"]
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device="cuda")
        C_col = torch.empty(F, dtype=torch.int32, device="cuda")
        C_val = torch.empty(F, dtype=torch.float64, device="cuda")
        nnz = binding.spgemm_compute(plan, a.val, b.val, C_rp, C_col, C_val)
        R = oracle.spgemm(A, B)
        W = np.random.default_rng(5).standard_normal(nnz)
        dA = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
        dB = torch.empty(B.nnz, dtype=torch.float64, device="cuda")
        binding.spgemm_backward(plan, a.val, b.val, torch.from_numpy(W).cuda(), dA, dB, tws)
        binding.spgemm_status(plan)
    finally:
        binding.spgemm_free(plan)
    gA, gB = oracle.grad(A, B, R, W)
    Aa, Ba = A.copy(), B.copy()                   # error scale: the same sums over absolute values
    Aa.val, Ba.val = np.abs(A.val), np.abs(B.val)
    sA, sB = oracle.grad(Aa, Ba, R, np.abs(W))
    if layout.startswith("csc"):
        gA, sA = to_csc_order(A, gA), to_csc_order(A, sA)
    if layout.endswith("csc"):
        gB, sB = to_csc_order(B, gB), to_csc_order(B, sB)
    for got, ref, sc in ((dA.cpu().numpy(), gA, sA), (dB.cpu().numpy(), gB, sB)):
        err = np.abs(got - ref) / np.where(sc > 0, sc, 1.0)
        assert err.max(initial=0.0) <= 1e-12


def test_validate_checks_csc_indices():
    A = synth.random_k(400, 3, 431, ncols=300)
    a = dev_csc(A)
    a.row_idx[17] = 400                            # a row index past the last row
    b = binding.DeviceCSR.from_host(synth.random_k(300, 3, 432))
    opt = binding.with_storage(a, b, binding.options(validate=1))
    ws = torch.empty(binding.spgemm_workspace_size(a, b, opt), dtype=torch.uint8, device="cuda")
    with pytest.raises(binding.SpgemmError, match="INVALID"):
        binding.spgemm_plan(a, b, ws, opt)


# ---- torch front door ------------------------------------------------------------------------

def torch_csr(M):
    return torch.sparse_csr_tensor(torch.from_numpy(np.asarray(M.row_ptr, np.int32)).cuda(),
                                   torch.from_numpy(np.asarray(M.col_idx, np.int32)).cuda(),
                                   torch.from_numpy(np.asarray(M.val, np.float64)).cuda(), size=(M.rows, M.cols))


def torch_csc(M):
    cp, ri, v = oracle.transpose(M)
    return torch.sparse_csc_tensor(torch.from_numpy(cp.astype(np.int32)).cuda(),
                                   torch.from_numpy(ri.astype(np.int32)).cuda(),
                                   torch.from_numpy(v).cuda(), size=(M.rows, M.cols))


def from_torch(C):
    return dict(row_ptr=C.crow_indices().cpu().numpy(), col_idx=C.col_indices().cpu().numpy(),
                val=C.values().cpu().numpy())


@pytest.mark.parametrize("layout", ["csr-csr", "csr-csc", "csc-csr", "csc-csc"])
def test_torch_spgemm(layout):
    from paper_1303_1651_gb300 import spgemm
    A = synth.random_k(900, 6, 441, ncols=700)
    B = synth.random_k(700, 7, 442, ncols=1100)
    tA = torch_csc(A) if layout.startswith("csc") else torch_csr(A)
    tB = torch_csc(B) if layout.endswith("csc") else torch_csr(B)
    C = spgemm(tA, tB)
    assert C.layout == torch.sparse_csr and C.shape == (900, 1100)
    assert C.crow_indices().dtype == torch.int32 and C.values().dtype == torch.float64
    compare(from_torch(C), oracle.spgemm(A, B), single=True)


def test_torch_spgemm_laplacian_and_empty():
    from paper_1303_1651_gb300 import spgemm
    L = synth.laplacian5(30)
    compare(from_torch(spgemm(torch_csr(L), torch_csr(L))), oracle.spgemm(L, L), exact=True)
    # no rows, and no entries
    E = synth.CSR(0, 50, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = synth.random_k(50, 3, 443, ncols=60)
    C = spgemm(torch_csr(E), torch_csr(B))
    assert C.shape == (0, 60) and C.values().numel() == 0
    Z = synth.CSR(20, 50, np.zeros(21, np.int32), np.zeros(0, np.int32), np.zeros(0))
    C = spgemm(torch_csr(Z), torch_csc(B))
    assert C.shape == (20, 60) and C.values().numel() == 0 and int(C.crow_indices().abs().sum()) == 0


def test_torch_spgemm_rejects_wrong_inputs():
    from paper_1303_1651_gb300 import spgemm
    A = synth.random_k(40, 3, 451, ncols=30)
    B = synth.random_k(30, 3, 452, ncols=20)
    tA, tB = torch_csr(A), torch_csr(B)
    with pytest.raises(TypeError):
        spgemm(tA.to_dense(), tB)
    with pytest.raises(TypeError):
        spgemm(torch.sparse_csr_tensor(tA.crow_indices().long(), tA.col_indices().long(), tA.values(),
                                       size=tA.shape), tB)
    with pytest.raises(TypeError):
        spgemm(torch.sparse_csr_tensor(tA.crow_indices(), tA.col_indices(), tA.values().float(), size=tA.shape), tB)
    with pytest.raises(ValueError):
        spgemm(tB, tB)
