"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Pattern (row_ptr, col_idx) must match bit-exactly; values within 1e-12 of the
sum of |a*b| of the entry.  Merge-class rows sum in the oracle's order, so
their values are also compared bit-exactly."""
import numpy as np
import pytest

import oracle
from paper_1303_1651_gb300 import synth
from tests.gpu_util import compare, gpu_product

pytestmark = pytest.mark.gpu


def opts(**kw):
    from paper_1303_1651_gb300 import binding
    return binding.options(**kw)


def test_laplacian_64_squared():
    A = synth.laplacian5(64)
    C = gpu_product(A, A)
    R = oracle.spgemm(A, A)
    compare(C, R, exact=True)
    assert C["info"]["products"] == 100104 and C["nnz"] == 51972


def test_random_4096_k8():
    A, B = synth.random_k(4096, 8, synth.SEED_A), synth.random_k(4096, 8, synth.SEED_B)
    compare(gpu_product(A, B), oracle.spgemm(A, B), exact=True)


@pytest.mark.parametrize("k", [1, 2, 4, 5, 7, 8])
def test_random_merge_classes(k):
    A, B = synth.random_k(3000, k, 11 + k), synth.random_k(3000, k, 31 + k)
    C = gpu_product(A, B)
    compare(C, oracle.spgemm(A, B), exact=True)


@pytest.mark.parametrize("k", [9, 16, 32])
def test_random_hash_classes(k):
    A, B = synth.random_k(2000, k, 5 + k), synth.random_k(2000, k, 7 + k)
    C = gpu_product(A, B)
    compare(C, oracle.spgemm(A, B))
    assert C["info"]["rows_per_class"]["W"] + C["info"]["rows_per_class"]["B"] > 0


def test_power_law_all_classes():
    A = synth.power_law(3000, 3000, 3, alpha=1.5, max_len=3000)
    B = synth.power_law(3000, 4000, 4, alpha=1.5, max_len=400)
    C = gpu_product(A, B)
    R = oracle.spgemm(A, B)
    compare(C, R)
    cls = C["info"]["rows_per_class"]
    assert all(cls[c] > 0 for c in ("M1", "M2", "W", "B", "G")), cls


@pytest.mark.parametrize("forced", [
    dict(m1_max_u=-1, m2_max_u=-1),                                   # everything hashed
    dict(m1_max_u=-1, m2_max_u=-1, warp_max_u=-1),                    # block hash
    dict(m1_max_u=-1, m2_max_u=-1, warp_max_u=-1, block_max_u=-1),   # dense fallback only
    dict(m1_max_u=4, m2_max_u=16, warp_max_u=40, block_max_u=100, dense_slabs=3),
])
def test_forced_classes(forced):
    A = synth.power_law(1500, 1200, 8, alpha=1.7, max_len=300)
    B = synth.power_law(1200, 900, 9, alpha=1.7, max_len=100)
    compare(gpu_product(A, B, opts(**forced)), oracle.spgemm(A, B))


def test_laplacian_forced_classes_exact():
    A = synth.laplacian5(40)
    R = oracle.spgemm(A, A)
    for forced in (dict(m1_max_u=-1, m2_max_u=-1), dict(m1_max_u=-1, m2_max_u=-1, warp_max_u=-1, block_max_u=-1)):
        compare(gpu_product(A, A, opts(**forced)), R, exact=True)   # small integers: every order is exact


def test_rectangular_and_empty_rows():
    rng = np.random.default_rng(12)
    lengths = rng.integers(0, 20, size=700)
    lengths[100:200] = 0                        # a block of empty rows
    A = synth.random_lengths(lengths, 300, 12)  # 700 x 300
    blen = rng.integers(0, 25, size=300)
    blen[::7] = 0                               # empty rows of B as well
    B = synth.random_lengths(blen, 1100, 13)    # 300 x 1100
    compare(gpu_product(A, B), oracle.spgemm(A, B))


def test_degenerate_shapes():
    one = synth.from_dense(np.array([[2.5]]))
    C = gpu_product(one, one)
    assert list(C["val"]) == [6.25]
    Z = synth.CSR(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = synth.random_k(5, 2, 1)
    C = gpu_product(Z, B)
    assert C["nnz"] == 0 and list(C["row_ptr"]) == [0]
    E = synth.CSR(4, 5, np.zeros(5, np.int32), np.zeros(0, np.int32), np.zeros(0))
    C = gpu_product(E, B)
    assert C["nnz"] == 0 and list(C["row_ptr"]) == [0] * 5
    Bz = synth.CSR(5, 3, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0))
    A = synth.random_k(7, 2, 3, ncols=5)
    C = gpu_product(A, Bz)      # every B row empty
    assert C["nnz"] == 0


def test_cancellation_and_explicit_zeros():
    A = synth.CSR(1, 2, np.array([0, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, 1.0]))
    B = synth.CSR(2, 1, np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([1.0, -1.0]))
    C = gpu_product(A, B)
    assert C["nnz"] == 1 and C["val"][0] == 0.0
    Az = synth.random_k(500, 6, 3)
    Az.val[::3] = 0.0
    Bz = synth.random_k(500, 6, 4)
    Bz.val[::5] = 0.0
    compare(gpu_product(Az, Bz), oracle.spgemm(Az, Bz), exact=True)


def test_unsorted_A_and_duplicates_in_A():
    A = synth.duplicate_entries(synth.random_k(800, 5, 21), 22)   # unsorted rows with repeated columns
    B = synth.random_k(800, 6, 23)
    compare(gpu_product(A, B), oracle.spgemm(A, B))


def test_unsorted_B_reported_for_merge_rows_and_hashed_otherwise():
    from paper_1303_1651_gb300 import binding
    A = synth.random_k(600, 4, 31)
    B = synth.shuffle_rows(synth.random_k(600, 6, 32), 33)
    with pytest.raises(binding.SpgemmError) as e:
        gpu_product(A, B)
    assert e.value.name == "SPGEMM_ERR_UNSORTED"
    compare(gpu_product(A, B, opts(m1_max_u=-1, m2_max_u=-1)), oracle.spgemm(A, B))


def test_numeric_repeatable_with_new_values():
    from paper_1303_1651_gb300 import binding
    import torch
    A, B = synth.random_k(2000, 7, 41), synth.laplacian5(45)
    A = synth.random_k(2025, 7, 41)
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    prod = binding.Product(dA, dB)
    try:
        for t in range(3):
            A2 = A.copy(); A2.val = A.val * (t + 1) - t
            C = prod.numeric(A_val=torch.from_numpy(A2.val).cuda())
            binding.spgemm_status(prod.plan)
            out = C.to_host()
            compare(out, oracle.spgemm(A2, B), exact=True)
    finally:
        prod.close()


def test_validate_option_flags_bad_columns():
    from paper_1303_1651_gb300 import binding
    A = synth.random_k(100, 3, 51)
    B = synth.random_k(100, 3, 52)
    B.col_idx[5] = 1000       # out of range column in B
    with pytest.raises(binding.SpgemmError) as e:
        gpu_product(A, B, opts(validate=1))
    assert e.value.name == "SPGEMM_ERR_INVALID"
