"""spgemm_multiply: plan and single-pass product in one call with one host read-back, against the
CPU oracle (pattern bit-exact, values within 1e-12 of sum |a*b|, single-product entries bit-exact).

Its class kernels learn their row counts on the device, and both tile forms of the fused pass are
launched before the host knows which one the binning chose, so every class mix and both forms are
checked here, together with the capacity report (OVERFLOW with F, then a retry) and a workspace
reused across calls with different matrices (the dense accumulators start from uncleared memory)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1303_1651_gb300 import binding, synth
from tests.gpu_util import compare

pytestmark = pytest.mark.gpu


def dev(M):
    return binding.DeviceCSR.from_host(M)


def once(A, B, opt=None, capacity=None, workspace=None):
    C = binding.multiply_once(dev(A), dev(B) if B is not A else dev(A), opt, capacity=capacity, workspace=workspace)
    torch.cuda.synchronize()
    return C.to_host()


@pytest.mark.parametrize("case", ["lap64", "rand-k4", "rand-k8", "rect", "power-law", "dense-rows"])
def test_matches_oracle(case):
    if case == "lap64":
        A = synth.laplacian5(64)
        compare(once(A, A), oracle.spgemm(A, A), exact=True)
        return
    if case == "rand-k4":            # 32-product tiles
        A, B = synth.random_k(5000, 4, 501), synth.random_k(5000, 4, 502)
    elif case == "rand-k8":          # 64-product rows: the two-lanes-per-row form is the one that runs
        A, B = synth.random_k(5000, 8, 503), synth.random_k(5000, 8, 504)
    elif case == "rect":
        A, B = synth.random_k(1700, 6, 505, ncols=900), synth.random_k(900, 7, 506, ncols=2500)
    elif case == "power-law":        # every class at once
        A = synth.power_law(3000, 3000, 3, alpha=1.5, max_len=3000)
        B = synth.power_law(3000, 4000, 4, alpha=1.5, max_len=400)
    else:                            # the paper's 0.1 % fill rows: class B
        A, B = synth.random_fill(20_000, 0.003, 507), synth.random_fill(20_000, 0.003, 508)
    compare(once(A, B), oracle.spgemm(A, B), single=True)


@pytest.mark.parametrize("forced", [dict(m1_max_u=-1, m2_max_u=-1), dict(m1_max_u=-1, m2_max_u=-1, warp_max_u=-1),
                                    dict(m1_max_u=-1, m2_max_u=-1, warp_max_u=-1, block_max_u=-1),
                                    dict(merge_values=2), dict(merge_values=1, m2_max_u=32)],
                         ids=["warp", "block", "dense", "staged", "direct-32"])
def test_forced_classes(forced):
    A = synth.power_law(1500, 1200, 8, alpha=1.7, max_len=300)
    B = synth.power_law(1200, 900, 9, alpha=1.7, max_len=100)
    compare(once(A, B, binding.options(**forced)), oracle.spgemm(A, B))


def test_capacity_report_and_retry():
    A, B = synth.random_k(4000, 6, 511), synth.random_k(4000, 6, 512)
    R = oracle.spgemm(A, B)
    dA, dB = dev(A), dev(B)
    ws = torch.empty(binding.spgemm_workspace_size(dA, dB), dtype=torch.uint8, device="cuda")
    C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device="cuda")
    small = 1000
    C_col = torch.full((small + 64,), -7, dtype=torch.int32, device="cuda")
    C_val = torch.zeros(small + 64, dtype=torch.float64, device="cuda")
    nnz, F = binding.spgemm_multiply(dA, dB, C_rp, C_col[:small], C_val[:small], ws, raise_on_overflow=False)
    assert nnz == R["nnz"] and F == R["F"]
    torch.cuda.synchronize()
    assert bool((C_col[small:] == -7).all()), "written past the capacity"
    with pytest.raises(binding.SpgemmError, match="OVERFLOW"):
        binding.spgemm_multiply(dA, dB, C_rp, C_col[:small], C_val[:small], ws)
    # the product through the helper: one call that overflows, then one with C sized by F
    C = binding.multiply_once(dA, dB, capacity=small)
    torch.cuda.synchronize()
    compare(C.to_host(), R, single=True)


def test_workspace_reused_across_products():
    # one workspace for a sequence of products of different shapes, classes and sizes
    probs = [(synth.power_law(2000, 2000, 21, alpha=1.5, max_len=2000), synth.power_law(2000, 3000, 22, alpha=1.5,
                                                                                       max_len=500)),
             (synth.random_k(3000, 8, 23), synth.random_k(3000, 8, 24)),
             (synth.laplacian5(40), None),
             (synth.power_law(2000, 2000, 25, alpha=1.4, max_len=2000), synth.power_law(2000, 3000, 26, alpha=1.4,
                                                                                        max_len=500))]
    size = 0
    for A, B in probs:
        B = A if B is None else B
        size = max(size, binding.spgemm_workspace_size(dev(A), dev(B)))
    ws = torch.full((size,), 0xAB, dtype=torch.uint8, device="cuda")     # not cleared on purpose
    for A, B in probs:
        B = A if B is None else B
        compare(once(A, B, workspace=ws), oracle.spgemm(A, B))


def test_empty_and_csc():
    E = synth.CSR(0, 50, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = synth.random_k(50, 3, 521, ncols=60)
    C = once(E, B)
    assert C["rows"] == 0 and C["nnz"] == 0
    Z = synth.CSR(30, 50, np.zeros(31, np.int32), np.zeros(0, np.int32), np.zeros(0))
    C = once(Z, B)
    assert C["nnz"] == 0 and not C["row_ptr"].any()
    # B given in compressed columns
    A = synth.random_k(800, 5, 522, ncols=600)
    Bc = synth.random_k(600, 6, 523, ncols=700)
    cp, ri, v = oracle.transpose(Bc)
    b = binding.DeviceCSC(Bc.rows, Bc.cols, torch.from_numpy(cp.astype(np.int32)).cuda(),
                          torch.from_numpy(ri.astype(np.int32)).cuda(), torch.from_numpy(v).cuda())
    C = binding.multiply_once(dev(A), b)
    torch.cuda.synchronize()
    compare(C.to_host(), oracle.spgemm(A, Bc), single=True)


@pytest.mark.parametrize("case", ["rand-k6", "power-law"])
def test_graph_replay(case):
    # spgemm_multiply_async captured once into a CUDA graph, replayed over new contents of the same
    # arrays: new values, then a new pattern of the same sizes (other row classes, another nnz(C))
    if case == "rand-k6":
        mats = [(synth.random_k(6000, 6, 531 + 2 * i), synth.random_k(6000, 6, 532 + 2 * i)) for i in range(3)]
    else:
        mats = [(synth.power_law(2500, 2500, 41 + 2 * i, alpha=1.5, max_len=2500),
                 synth.power_law(2500, 3000, 42 + 2 * i, alpha=1.5, max_len=600)) for i in range(3)]
    # the same nnz for each operand in every product: the patterns are cut or padded to the first's
    def fit(M, nnz):
        rp = np.minimum(M.row_ptr.astype(np.int64), nnz)
        col = M.col_idx[:nnz]
        val = M.val[:nnz]
        if len(col) < nnz:                          # pad the last row with repeated columns
            pad = nnz - len(col)
            col = np.concatenate([col, np.full(pad, M.cols - 1, np.int32)])
            val = np.concatenate([val, np.full(pad, 0.5)])
        rp[-1] = nnz
        return synth.CSR(M.rows, M.cols, rp.astype(np.int32), col.astype(np.int32), val)
    nA, nB = mats[0][0].nnz, mats[0][1].nnz
    mats = [(fit(A, nA), fit(B, nB)) for A, B in mats]
    dA, dB = dev(mats[0][0]), dev(mats[0][1])
    cap = max(oracle.spgemm(A, B)["nnz"] for A, B in mats)
    g = binding.GraphProduct(dA, dB, cap)
    for i, (A, B) in enumerate(mats):
        R = oracle.spgemm(A, B)
        for X, dX in ((A, dA), (B, dB)):
            dX.row_ptr.copy_(torch.from_numpy(X.row_ptr))
            dX.col_idx.copy_(torch.from_numpy(X.col_idx))
            dX.val.copy_(torch.from_numpy(X.val))
        for rep in range(2):                        # a second replay gives the same C
            nnz, F = g.run()
            assert (nnz, F) == (R["nnz"], R["F"]), (i, rep)
            got = dict(row_ptr=g.C_row_ptr.cpu().numpy(), col_idx=g.C_col[:nnz].cpu().numpy(),
                       val=g.C_val[:nnz].cpu().numpy())
            compare(got, R, single=True)
        # with new values only: the numbers change, the pattern does not
        dA.val.mul_(-2.0)
        nnz, _ = g.run()
        R2 = oracle.spgemm(synth.CSR(A.rows, A.cols, A.row_ptr, A.col_idx, -2.0 * A.val), B)
        compare(dict(row_ptr=g.C_row_ptr.cpu().numpy(), col_idx=g.C_col[:nnz].cpu().numpy(),
                     val=g.C_val[:nnz].cpu().numpy()), R2, single=True)


def test_graph_replay_overflow_report():
    A, B = synth.random_k(3000, 6, 541), synth.random_k(3000, 6, 542)
    R = oracle.spgemm(A, B)
    g = binding.GraphProduct(dev(A), dev(B), R["nnz"] // 2)
    with pytest.raises(binding.SpgemmError, match="OVERFLOW"):
        g.run()
    assert g.run(raise_on_overflow=False) == (R["nnz"], R["F"])


def test_invalid_entry_reported_without_fault():
    # a column of A outside B's rows: the binning pass gives its row no class, so no kernel of the
    # one-call product addresses B's row pointer with it; the call reports INVALID, and the device
    # is exact on the next product
    A, B = synth.random_k(2000, 5, 551), synth.random_k(2000, 5, 552)
    bad = synth.CSR(A.rows, A.cols, A.row_ptr.copy(), A.col_idx.copy(), A.val.copy())
    bad.col_idx[777] = B.rows + 5
    dA, dB = dev(bad), dev(B)
    ws = torch.empty(binding.spgemm_workspace_size(dA, dB), dtype=torch.uint8, device="cuda")
    F = int(oracle.spgemm(A, B)["F"])
    C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device="cuda")
    C_col = torch.empty(F, dtype=torch.int32, device="cuda")
    C_val = torch.empty(F, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.SpgemmError, match="INVALID"):
        binding.spgemm_multiply(dA, dB, C_rp, C_col, C_val, ws)
    torch.cuda.synchronize()
    compare(once(A, B), oracle.spgemm(A, B))
