"""The size sweep's recipe and its size-independent checks, on the CPU: the checks the GPU sweep
test applies must accept a correct product and reject planted mistakes, the device form of the
Laplacian² closed form must equal the geometric one of the oracle pins, and the oracle's product
of a row sample must equal those rows of the whole product."""
import numpy as np
import pytest
import torch

import oracle
from paper_1303_1651_gb300 import synth
from tests import pins
from tests.sweep_util import (check_structure, gpu_rows, laplacian_square, products_count, ranges, sample_rows,
                              sub_problem)


def test_sweep_points_recipe():
    pts = synth.sweep_points()
    assert len(pts) == 52
    sizes = synth.sweep_sizes()
    assert sizes[0] == 1000 and sizes[-1] == 10_000_000 and sizes[3] == 10_000 and sizes[6] == 100_000
    assert sizes == sorted(sizes) and all(abs(np.log10(b / a) - 1 / 3) < 1e-3 for a, b in zip(sizes, sizes[1:]))
    A, B = synth.sweep_problem(2154, "lap")
    assert A is B and A.rows == 46 * 46
    A, B = synth.sweep_problem(2154, "rand8")
    assert A.rows == A.cols == B.rows == 2154 and A.nnz == B.nnz == 8 * 2154
    assert not np.array_equal(A.col_idx, B.col_idx)
    for M in (A, B):     # k distinct columns per row
        rows = np.repeat(np.arange(M.rows), 8)
        assert len(set(zip(rows.tolist(), M.col_idx.tolist()))) == M.nnz
    with pytest.raises(ValueError):
        synth.sweep_problem(1000, "band")


@pytest.mark.parametrize("n", [5, 8, 33])
def test_laplacian_square_device_form_equals_geometry(n):
    rp, col, val = laplacian_square(n, device="cpu")
    E = pins.laplacian_square_closed_form(n)
    assert np.array_equal(rp.numpy(), E["row_ptr"])
    assert np.array_equal(col.numpy(), E["col_idx"])
    assert np.array_equal(val.numpy(), E["val"])


def _as_tensors(R):
    return (torch.from_numpy(np.asarray(R["row_ptr"], np.int32)), torch.from_numpy(np.asarray(R["col_idx"], np.int32)),
            torch.from_numpy(np.asarray(R["val"])))


def test_structure_check_accepts_and_rejects():
    A, B = synth.sweep_problem(4642, "rand4")
    R = oracle.spgemm(A, B)
    rp, col, _ = _as_tensors(R)
    nnz = int(R["nnz"])
    check_structure(rp, col, nnz, B.cols)
    assert products_count(A, B) == R["F"] == oracle.flops(A, B)
    s = int(rp[100])
    swapped = col.clone()
    swapped[s], swapped[s + 1] = col[s + 1], col[s]
    dup = col.clone()
    dup[s + 1] = col[s]
    out = col.clone()
    out[-1] = B.cols
    bad_rp = rp.clone()
    bad_rp[50] = bad_rp[52]
    for c, r, why in ((swapped, rp, "swapped columns"), (dup, rp, "repeated column"), (out, rp, "column out of range"),
                      (col, bad_rp, "row pointer decreases")):
        with pytest.raises(AssertionError):
            check_structure(r, c, nnz, B.cols)
            pytest.fail(why)
    with pytest.raises(AssertionError):
        check_structure(rp, col, nnz - 1, B.cols)


@pytest.mark.parametrize("kind", ["rand4", "rand16"])
def test_row_sample_equals_rows_of_the_whole_product(kind):
    A, B = synth.sweep_problem(4642, kind)
    R = oracle.spgemm(A, B)
    rows = sample_rows(A.rows, seed=3, count=200)
    assert rows[0] == 0 and rows[-1] == A.rows - 1 and np.all(np.diff(rows) > 0)
    A_sub, B_sub = sub_problem(A, B, rows)
    S = oracle.spgemm(A_sub, B_sub)
    got = gpu_rows(*_as_tensors(R), rows, B.cols)
    assert np.array_equal(got["row_ptr"], S["row_ptr"])
    assert np.array_equal(got["col_idx"].astype(np.int64), S["col_idx"])
    assert np.array_equal(got["val"].view(np.int64), S["val"].view(np.int64))


def test_ranges():
    assert ranges(np.array([5, 0, 9, 4]), np.array([5, 3, 11, 6])).tolist() == [0, 1, 2, 9, 10, 4, 5]
    assert ranges(np.array([], np.int64), np.array([], np.int64)).tolist() == []
