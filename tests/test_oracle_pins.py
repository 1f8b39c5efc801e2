"""Pins for the CPU oracle (no GPU): dense products, closed forms, invariants,
exact finite differences, and planted mistakes that each pin must catch."""
import numpy as np
import pytest

import oracle
from paper_1303_1651_gb300 import synth
from tests import pins


def tiny_problem(seed, m=None, k=None, n=None, density=0.25):
    rng = np.random.default_rng(seed)
    m = m or int(rng.integers(1, 24))
    k = k or int(rng.integers(1, 24))
    n = n or int(rng.integers(1, 24))
    def mat(r, c):
        mask = rng.random((r, c)) < density
        vals = rng.integers(-3, 4, size=(r, c)).astype(float)
        vals[vals == 0] = 2.0
        return synth.from_dense(np.where(mask, vals, 0.0))
    return mat(m, k), mat(k, n)


@pytest.mark.parametrize("seed", range(12))
def test_dense_product_pin(seed):
    A, B = tiny_problem(seed)
    pins.check_dense_product(oracle.spgemm, A, B)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 64])
def test_laplacian_square_closed_form(n):
    pins.check_laplacian_square(oracle.spgemm, n)


def test_laplacian_square_large_counts():
    # the 64 x 64 grid case, and the published counts of the 2048 grid via the formulas
    A = synth.laplacian5(64)
    C = oracle.spgemm(A, A)
    assert (C["nnz"], C["F"]) == (51972, 100104)
    n = 2048
    assert 13 * n * n - 20 * n + 4 == 54484996
    assert 25 * (n - 2) ** 2 + 64 * (n - 2) + 36 == 104783880


def test_cancellation_kept():
    pins.check_cancellation(oracle.spgemm)


def test_explicit_zero_is_structural():
    A = synth.from_dense(np.array([[0.0, 2.0]]), keep_zeros_mask=np.array([[True, True]]))
    B = synth.from_dense(np.array([[5.0, 0.0], [0.0, 3.0]]))
    C = oracle.spgemm(A, B)
    assert list(C["col_idx"]) == [0, 1] and list(C["val"]) == [0.0, 6.0]


def test_flop_formula_matches_row_counts():
    # Section III counts multiplications by columns of A and rows of B; the oracle's
    # row loop counts them per row of A.  Two different sums must agree.
    for seed in range(5):
        A = synth.power_law(300, 200, seed, max_len=60)
        B = synth.power_law(200, 150, seed + 100, max_len=40)
        C = oracle.spgemm(A, B)
        assert C["F"] == int(C["u"].sum()) == oracle.flops(A, B)
        assert C["nnz"] <= C["F"]      # the never-underestimating estimate of Section IV-B
        pins.check_csr_invariants(C)


def test_entry_product_counts():
    # every multiplication lands in exactly one entry; the Laplacian^2 diagonal gathers 1 + deg products
    A = synth.power_law(200, 150, 31, max_len=30)
    B = synth.power_law(150, 170, 32, max_len=20)
    C = oracle.spgemm(A, B)
    assert int(C["count"].sum()) == C["F"] and C["count"].min(initial=1) >= 1
    n = 6
    L = synth.laplacian5(n)
    C = oracle.spgemm(L, L)
    for i in range(n):
        for j in range(n):
            r = i * n + j
            seg = slice(C["row_ptr"][r], C["row_ptr"][r + 1])
            diag = np.nonzero(C["col_idx"][seg] == r)[0][0]
            deg = (i > 0) + (i < n - 1) + (j > 0) + (j < n - 1)
            assert C["count"][seg][diag] == 1 + deg


def test_row_counts_are_products_per_row():
    A = synth.random_k(500, 6, 1)
    B = synth.power_law(500, 400, 2, max_len=30)
    C = oracle.spgemm(A, B)
    blen = np.diff(B.row_ptr)
    u = np.array([blen[A.col_idx[A.row_ptr[r]:A.row_ptr[r + 1]]].sum() for r in range(A.rows)])
    assert np.array_equal(u, C["u"])


def test_random_nnz_statistics():
    # not a gate: the expected distinct-column count of k^2 uniform draws in N columns
    N, k = 20000, 8
    A, B = synth.random_k(N, k, synth.SEED_A), synth.random_k(N, k, synth.SEED_B)
    C = oracle.spgemm(A, B)
    expect = N * N * (1 - (1 - 1 / N) ** (k * k))
    assert abs(C["nnz"] - expect) / expect < 1e-3


def test_unsorted_and_duplicate_inputs():
    A = synth.integer_valued(synth.power_law(80, 60, 3, max_len=20), 4)
    B = synth.integer_valued(synth.power_law(60, 70, 5, max_len=20), 6)
    base = oracle.spgemm(A, B)
    for As, Bs in [(synth.shuffle_rows(A, 7), B), (A, synth.shuffle_rows(B, 8)),
                   (synth.shuffle_rows(A, 9), synth.shuffle_rows(B, 10))]:
        C = oracle.spgemm(As, Bs)
        assert np.array_equal(C["row_ptr"], base["row_ptr"]) and np.array_equal(C["col_idx"], base["col_idx"])
        assert np.array_equal(C["val"], base["val"])  # integer values: exact in any order
    Ad = synth.integer_valued(synth.duplicate_entries(A, 11), 12)
    pins.check_dense_product(oracle.spgemm, Ad, B)


def test_gradients_dense_and_finite_difference():
    A, B = tiny_problem(21, 15, 12, 18, density=0.3)
    C = oracle.spgemm(A, B)
    rng = np.random.default_rng(5)
    W = rng.integers(-4, 5, size=C["nnz"]).astype(float)
    dA, dB = oracle.grad(A, B, C, W)
    Wd = np.zeros((A.rows, B.cols))
    r = np.repeat(np.arange(A.rows), np.diff(C["row_ptr"]))
    Wd[r, C["col_idx"]] = W
    GA = Wd @ B.to_dense().T
    GB = A.to_dense().T @ Wd
    ra = np.repeat(np.arange(A.rows), np.diff(A.row_ptr))
    rb = np.repeat(np.arange(B.rows), np.diff(B.row_ptr))
    assert np.array_equal(dA, GA[ra, A.col_idx])
    assert np.array_equal(dB, GB[rb, B.col_idx])
    # the loss is affine in each single entry: a unit step changes it by exactly the gradient
    def loss(A_, B_):
        C_ = oracle.spgemm(A_, B_)
        return float((pins.dense_of(C_) * Wd).sum())
    L0 = loss(A, B)
    for p in range(0, A.nnz, 7):
        A2 = A.copy(); A2.val[p] += 1.0
        assert loss(A2, B) - L0 == dA[p]
    for q in range(0, B.nnz, 7):
        B2 = B.copy(); B2.val[q] += 1.0
        assert loss(A, B2) - L0 == dB[q]


def test_transpose():
    A = synth.power_law(40, 30, 9, max_len=10)
    cp, ri, tv = oracle.transpose(A)
    D = A.to_dense().T
    T = synth.CSR(A.cols, A.rows, cp.astype(np.int32), ri.astype(np.int32), tv)
    assert np.array_equal(T.to_dense(), D)
    for c in range(A.cols):
        assert np.all(np.diff(ri[cp[c]:cp[c + 1]]) > 0)


def test_empty_and_degenerate():
    Z = synth.CSR(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = synth.random_k(5, 2, 1)
    C = oracle.spgemm(Z, B)
    assert C["nnz"] == 0 and len(C["row_ptr"]) == 1
    E = synth.CSR(3, 5, np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0))
    C = oracle.spgemm(E, B)
    assert C["nnz"] == 0 and list(C["row_ptr"]) == [0, 0, 0, 0]
    one = synth.from_dense(np.array([[2.5]]))
    C = oracle.spgemm(one, one)
    assert list(C["val"]) == [6.25]


# ---- planted mistakes: every pin must reject a plausible bug --------------------------

def _mut_transposed_B(A, B):
    cp, ri, tv = oracle.transpose(B)
    Bt = synth.CSR(B.cols, B.rows, cp.astype(np.int32), ri.astype(np.int32), tv)
    if Bt.rows != A.cols:     # shape mismatch: fall back to a wrong but shaped product
        return _mut_sign(A, B)
    return oracle.spgemm(A, Bt)


def _mut_dropped_term(A, B):
    B2 = B.copy()
    if B2.nnz:
        B2.val[B2.nnz // 2] = 0.0   # one product dropped (pattern kept)
    return oracle.spgemm(A, B2)


def _mut_sign(A, B):
    C = oracle.spgemm(A, B)
    if C["nnz"]:
        C["val"][C["nnz"] // 3] *= -1
    return C


def _mut_drop_zero(A, B):
    C = oracle.spgemm(A, B)
    keep = C["val"] != 0.0
    rows = np.repeat(np.arange(C["rows"]), np.diff(C["row_ptr"]))[keep]
    C["row_ptr"] = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=C["rows"]))])
    C["col_idx"], C["val"], C["nnz"] = C["col_idx"][keep], C["val"][keep], int(keep.sum())
    return C


def _mut_unsorted(A, B):
    C = oracle.spgemm(A, B)
    rp = C["row_ptr"]
    for r in range(C["rows"]):
        if rp[r + 1] - rp[r] >= 2:
            a, b = rp[r], rp[r] + 1
            C["col_idx"][[a, b]] = C["col_idx"][[b, a]]
            C["val"][[a, b]] = C["val"][[b, a]]
            break
    return C


@pytest.mark.parametrize("mutant", [_mut_transposed_B, _mut_dropped_term, _mut_sign, _mut_unsorted])
def test_dense_pin_catches(mutant):
    caught = 0
    for seed in range(6):
        A, B = tiny_problem(100 + seed, 10, 10, 10, density=0.35)
        try:
            pins.check_dense_product(mutant, A, B)
        except AssertionError:
            caught += 1
    assert caught > 0


@pytest.mark.parametrize("mutant", [_mut_dropped_term, _mut_sign, _mut_unsorted])
def test_laplacian_pin_catches(mutant):
    with pytest.raises(AssertionError):
        pins.check_laplacian_square(mutant, 5)


def test_cancellation_pin_catches():
    with pytest.raises(AssertionError):
        pins.check_cancellation(_mut_drop_zero)
