"""Pattern reuse (spgemm_replay_record / spgemm_replay) through the C ABI.

With new values of A and B and the structures kept, replay must give C's values within the usual
tolerance of the oracle, and on the rows of the sort classes bit for bit equal to spgemm_numeric's
with the same values (both accumulate each entry in the loop order of the row-major algorithm)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1303_1651_gb300 import binding, synth
from tests.gpu_util import compare

pytestmark = pytest.mark.gpu


def new_values(M, seed):
    M2 = M.copy()
    M2.val = np.random.default_rng(seed).uniform(-1.0, 1.0, M.val.shape)
    return M2


def short_row_entries(A, B, C_row_ptr):
    """Mask of C's entries in rows of the sort classes (<= 8 entries of A, <= 64 products): the rows
    whose sums have a fixed order on both paths.  Longer rows use atomics (order not fixed)."""
    k = np.diff(A.row_ptr)
    blen = np.diff(B.row_ptr)
    r = np.repeat(np.arange(A.rows), k)
    u = np.bincount(r, weights=blen[A.col_idx], minlength=A.rows)
    short = (k <= 8) & (u <= 64)
    return np.repeat(short, np.diff(np.asarray(C_row_ptr, np.int64)))


def check_replay(A, B, opt=None, rounds=2, fused_first=False):
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    prod = binding.Product(dA, dB, opt)
    try:
        if fused_first:
            # record after the single-pass product instead of the three-call numeric
            F = max(prod.info["products"], 1)
            C_col = torch.empty(F, dtype=torch.int32, device="cuda")
            C_val = torch.empty(F, dtype=torch.float64, device="cuda")
            nnz = binding.spgemm_compute(prod.plan, dA.val, dB.val, prod.C_row_ptr, C_col, C_val)
            assert nnz == prod.nnz
            C = binding.DeviceCSR(A.rows, B.cols, prod.C_row_ptr, C_col[:nnz], C_val[:nnz])
        else:
            C = prod.numeric()
        prod.record(C)
        for t in range(rounds):
            A2, B2 = new_values(A, 100 + t), new_values(B, 200 + t)
            a2, b2 = torch.from_numpy(A2.val).cuda(), torch.from_numpy(B2.val).cuda()
            R = prod.replay(a2, b2)
            Rv = R.val.clone()
            N = prod.numeric(A_val=a2, B_val=b2)
            binding.spgemm_status(prod.plan)
            assert torch.equal(R.col_idx, N.col_idx)
            mask = short_row_entries(A, B, prod.C_row_ptr.cpu().numpy())
            rb, nb = Rv.view(torch.int64).cpu().numpy(), N.val.view(torch.int64).cpu().numpy()
            assert np.array_equal(rb[mask], nb[mask]), "replay differs from numeric on short rows"
            out = R.to_host()
            out["val"] = Rv.cpu().numpy()
            compare(out, oracle.spgemm(A2, B2), single=True)
    finally:
        prod.close()


def test_replay_laplacian():
    L = synth.laplacian5(40)
    check_replay(L, L)


@pytest.mark.parametrize("k", [1, 3, 5, 8])
def test_replay_random(k):
    check_replay(synth.random_k(2500, k, 61 + k), synth.random_k(2500, k, 71 + k))


def test_replay_power_law_all_classes():
    A = synth.power_law(3000, 3000, 3, alpha=1.5, max_len=3000)
    B = synth.power_law(3000, 4000, 4, alpha=1.5, max_len=400)
    check_replay(A, B)


def test_replay_unsorted_and_duplicates():
    A = synth.duplicate_entries(synth.shuffle_rows(synth.random_k(1500, 4, 81), 82), 83)
    B = synth.shuffle_rows(synth.random_k(1500, 6, 84), 85)
    check_replay(A, B)


def test_replay_after_fused_product():
    check_replay(synth.random_k(3000, 8, 91), synth.random_k(3000, 8, 92), fused_first=True)
    L = synth.laplacian5(33)
    check_replay(L, L, fused_first=True)


def test_replay_value_modes():
    L = synth.laplacian5(30)
    for mode in (1, 2):
        check_replay(L, L, opt=binding.options(merge_values=mode), rounds=1)


def test_replay_errors():
    A, B = synth.random_k(500, 4, 95), synth.random_k(500, 4, 96)
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    prod = binding.Product(dA, dB)
    lib = binding.load()
    try:
        C = prod.numeric()
        size = binding.spgemm_replay_size(prod.plan)
        buf = torch.empty(size + 256, dtype=torch.uint8, device="cuda")
        # no map recorded yet
        assert lib.spgemm_replay(prod.plan, dA.val.data_ptr(), dB.val.data_ptr(), buf.data_ptr(),
                                 C.col_idx.data_ptr(), C.val.data_ptr(), None) == 7
        # too small, misaligned
        assert lib.spgemm_replay_record(prod.plan, C.col_idx.data_ptr(), buf.data_ptr(), size - 1, None) == 2
        assert lib.spgemm_replay_record(prod.plan, C.col_idx.data_ptr(), buf.data_ptr() + 16, size, None) == 1
        prod.record(C)
        # another buffer than the recorded map
        assert lib.spgemm_replay(prod.plan, dA.val.data_ptr(), dB.val.data_ptr(), buf.data_ptr(),
                                 C.col_idx.data_ptr(), C.val.data_ptr(), None) == 7
    finally:
        prod.close()
    # a C whose columns are not this product's: the record reports a mismatch
    prod = binding.Product(dA, dB)
    try:
        C = prod.numeric()
        wrong = (C.col_idx + 1) % B.cols
        buf = torch.empty(binding.spgemm_replay_size(prod.plan), dtype=torch.uint8, device="cuda")
        code = lib.spgemm_replay_record(prod.plan, wrong.data_ptr(), buf.data_ptr(), buf.numel(), None)
        assert code == 9, binding.error_string(code)
    finally:
        prod.close()


def test_replay_full_size_products():
    """The bench's products: replay equals numeric bit for bit with new values."""
    for A, B in ((synth.laplacian5(2048), None),
                 (synth.random_k(1_000_000, 8, synth.SEED_A), synth.random_k(1_000_000, 8, synth.SEED_B))):
        dA = binding.DeviceCSR.from_host(A)
        dB = dA if B is None else binding.DeviceCSR.from_host(B)
        prod = binding.Product(dA, dB)
        try:
            C = prod.numeric()
            prod.record(C)
            g = torch.Generator(device="cuda").manual_seed(5)
            a2 = torch.rand(dA.nnz, dtype=torch.float64, device="cuda", generator=g) * 2 - 1
            b2 = a2 if B is None else torch.rand(dB.nnz, dtype=torch.float64, device="cuda", generator=g) * 2 - 1
            R = prod.replay(a2, b2).val.clone()
            N = prod.numeric(A_val=a2, B_val=b2).val
            binding.spgemm_status(prod.plan)
            assert torch.equal(R.view(torch.int64), N.view(torch.int64))
        finally:
            prod.close()
