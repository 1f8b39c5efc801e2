"""Backward on the GPU: dA = (dC B^T) on A's structure, dB = (A^T dC) on B's structure,
against the oracle's gradient, finite differences, and torch.autograd.gradcheck."""
import numpy as np
import pytest
import torch

import oracle
from paper_1303_1651_gb300 import autograd, binding, synth

pytestmark = pytest.mark.gpu


def run_backward(A, B, W):
    dA_, dB_ = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    ws = torch.empty(binding.spgemm_workspace_size(dA_, dB_), dtype=torch.uint8, device="cuda")
    plan = binding.spgemm_plan(dA_, dB_, ws)
    try:
        F = max(binding.spgemm_plan_info(plan)["products"], 1)
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device="cuda")
        C_col = torch.empty(F, dtype=torch.int32, device="cuda")
        C_val = torch.empty(F, dtype=torch.float64, device="cuda")
        nnz = binding.spgemm_compute(plan, dA_.val, dB_.val, C_rp, C_col, C_val)
        assert nnz == W.size
        dW = torch.from_numpy(W).cuda()
        gA = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
        gB = torch.empty(B.nnz, dtype=torch.float64, device="cuda")
        tws = torch.empty(binding.spgemm_backward_workspace_size(dA_, dB_), dtype=torch.uint8, device="cuda")
        binding.spgemm_backward(plan, dA_.val, dB_.val, dW, gA, gB, tws)
        binding.spgemm_status(plan)
        # a second call reuses the transpose kept in the workspace
        gB2 = torch.empty_like(gB)
        binding.spgemm_backward(plan, dA_.val, dB_.val, dW, None, gB2, tws)
        binding.spgemm_status(plan)
        assert torch.equal(gB, gB2)
        return gA.cpu().numpy(), gB.cpu().numpy()
    finally:
        binding.spgemm_free(plan)


def check_grads(A, B, seed, tol=1e-12):
    C = oracle.spgemm(A, B)
    rng = np.random.default_rng(seed)
    W = rng.standard_normal(C["nnz"])
    gA, gB = run_backward(A, B, W)
    rA, rB = oracle.grad(A, B, C, W)
    # scale: the same sums over absolute values
    Aa, Ba = A.copy(), B.copy()
    Aa.val, Ba.val = np.abs(A.val), np.abs(B.val)
    sA, sB = oracle.grad(Aa, Ba, C, np.abs(W))
    for g, r, sc in ((gA, rA, sA), (gB, rB, sB)):
        err = np.abs(g - r) / np.where(sc > 0, sc, 1.0)
        assert err.max(initial=0.0) <= tol, err.max()
    return C, W, gA, gB


def test_backward_small_random_times_laplacian():
    A = synth.random_k(900, 16, 5, ncols=30 * 30)
    B = synth.laplacian5(30)
    check_grads(A, B, 1)


def test_backward_power_law_all_classes_and_empty_rows():
    rng = np.random.default_rng(2)
    la = rng.integers(0, 40, size=500); la[::9] = 0
    A = synth.random_lengths(la, 400, 3)
    lb = rng.integers(0, 30, size=400); lb[::7] = 0
    B = synth.random_lengths(lb, 600, 4)
    check_grads(A, B, 2)


def test_backward_finite_differences_exact_on_integers():
    A = synth.integer_valued(synth.random_k(60, 4, 7, ncols=50), 8)
    B = synth.integer_valued(synth.random_k(50, 3, 9, ncols=70), 10)
    C = oracle.spgemm(A, B)
    W = np.random.default_rng(3).integers(-3, 4, size=C["nnz"]).astype(float)
    gA, gB = run_backward(A, B, W)

    def loss(A_, B_):
        C_ = oracle.spgemm(A_, B_)
        return float(np.dot(C_["val"], W))   # same structure, entries aligned
    L0 = loss(A, B)
    for p in range(0, A.nnz, 5):
        A2 = A.copy(); A2.val[p] += 1.0
        assert loss(A2, B) - L0 == gA[p]
    for q in range(0, B.nnz, 5):
        B2 = B.copy(); B2.val[q] += 1.0
        assert loss(A, B2) - L0 == gB[q]


def test_autograd_gradcheck():
    A = synth.random_k(12, 3, 21, ncols=10)
    B = synth.random_k(10, 4, 22, ncols=9)
    dA_, dB_ = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    a = dA_.val.clone().requires_grad_(True)
    b = dB_.val.clone().requires_grad_(True)
    f = lambda x, y: autograd.spgemm(x, y, dA_, dB_)
    assert torch.autograd.gradcheck(f, (a, b), eps=1e-6, atol=1e-9)


def test_backward_full_size_random_times_laplacian():
    # A: 262144 x 262144, 16 distinct columns per row; B: Laplacian on a 512 x 512 grid
    A = synth.random_k(262144, 16, synth.SEED_A)
    B = synth.laplacian5(512)
    check_grads(A, B, synth.SEED_W)
