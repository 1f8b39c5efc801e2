"""The Combined CPU kernel (Section IV-B) against the oracle: same structure and, with the products
rounded on their own and added in the same loop order, the same values bit for bit, on one thread
and on several.  The per-row choice between the MinMax and the Sort store is checked against the
rule applied to the oracle's rows (range of the row's columns below twice its entry count)."""
import numpy as np
import pytest

import baseline
import oracle
from paper_1303_1651_gb300 import synth

THREADS = [1, 3, None]


def expected_minmax_rows(R) -> tuple[int, int]:
    """Rows the rule sends to MinMax and to Sort, from the oracle's C (empty rows go to neither)."""
    rp = np.asarray(R["row_ptr"], np.int64)
    lens = np.diff(rp)
    nz = lens > 0
    col = np.asarray(R["col_idx"], np.int64)
    first = col[rp[:-1][nz]]
    last = col[rp[1:][nz] - 1]
    minmax = (last - first + 1) < 2 * lens[nz]
    return int(minmax.sum()), int((~minmax).sum())


def check(A, B, threads):
    R = oracle.spgemm(A, B)
    C = baseline.combined(A, B, threads)
    assert C["F"] == R["F"]
    assert np.array_equal(C["row_ptr"], R["row_ptr"]), "row pointer differs"
    assert np.array_equal(C["col_idx"].astype(np.int64), R["col_idx"]), "columns differ"
    assert np.array_equal(C["val"].view(np.int64), R["val"].view(np.int64)), "values differ"
    assert (C["rows_minmax"], C["rows_sort"]) == expected_minmax_rows(R)
    return C


@pytest.mark.parametrize("threads", THREADS)
@pytest.mark.parametrize("n", [1, 2, 5, 6, 7, 40])
def test_laplacian_square(n, threads):
    A = synth.laplacian5(n)
    C = check(A, A, threads)
    if n == 6:       # interior rows: 13 entries over a range of 4n + 1 = 25 < 26 columns
        assert C["rows_minmax"] >= (n - 4) ** 2
    if n == 40:      # range 161 >= 26 on every interior row
        assert C["rows_sort"] >= (n - 4) ** 2


@pytest.mark.parametrize("threads", THREADS)
@pytest.mark.parametrize("N,k", [(20, 3), (64, 5), (3000, 1), (5000, 8), (2500, 16), (1200, 32)])
def test_random(N, k, threads):
    check(synth.random_k(N, k, 700 + k), synth.random_k(N, k, 800 + k), threads)


@pytest.mark.parametrize("threads", THREADS)
def test_power_law_and_rectangular(threads):
    check(synth.power_law(3000, 3000, 3, alpha=1.5, max_len=3000),
          synth.power_law(3000, 4000, 4, alpha=1.5, max_len=400), threads)
    check(synth.random_k(2100, 4, 11, ncols=900), synth.random_k(900, 6, 12, ncols=5000), threads)


@pytest.mark.parametrize("threads", THREADS)
def test_unsorted_duplicates_and_empty_rows(threads):
    A = synth.duplicate_entries(synth.shuffle_rows(synth.random_k(2500, 5, 21), 22), 23)
    B = synth.shuffle_rows(synth.random_k(2500, 7, 24), 25)
    check(A, B, threads)
    E = synth.random_lengths(np.where(np.arange(3000) % 3 == 0, 0, 4), 3000, 26)
    check(E, synth.random_k(3000, 4, 27), threads)
    check(synth.random_k(3000, 4, 28), E, threads)


def test_empty_and_cancellation():
    Z = synth.CSR(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    C = baseline.combined(Z, synth.random_k(5, 2, 1))
    assert C["nnz"] == 0 and list(C["row_ptr"]) == [0]
    A = synth.CSR(1, 2, np.array([0, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, 1.0]))
    B = synth.CSR(2, 1, np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([1.0, -1.0]))
    C = baseline.combined(A, B)
    assert C["nnz"] == 1 and list(C["col_idx"]) == [0] and C["val"][0] == 0.0


def test_bad_column_rejected():
    A = synth.random_k(50, 3, 1)
    B = synth.random_k(50, 3, 2)
    A.col_idx = A.col_idx.copy()
    A.col_idx[7] = 50
    with pytest.raises(ValueError):
        baseline.combined(A, B)
    A = synth.random_k(50, 3, 1)
    B.col_idx = B.col_idx.copy()
    B.col_idx[3] = -1
    with pytest.raises(ValueError):
        baseline.combined(A, B)
