"""Checks that pin a CSR product to facts other than the implementation itself.

Each ``check_*`` takes an implementation ``impl(A, B) -> dict`` (the oracle's
output format: row_ptr, col_idx, val, nnz, F) and raises AssertionError when
the implementation disagrees with the mathematics.  The tests apply them to the
oracle (must pass) and to planted mistakes (must fail).
"""
from __future__ import annotations

import numpy as np

from paper_1303_1651_gb300 import synth


def dense_of(C: dict) -> np.ndarray:
    D = np.zeros((C["rows"], C["cols"]))
    r = np.repeat(np.arange(C["rows"]), np.diff(C["row_ptr"]))
    np.add.at(D, (r, np.asarray(C["col_idx"], np.int64)), C["val"])
    return D


def pattern_of(C: dict) -> np.ndarray:
    P = np.zeros((C["rows"], C["cols"]), bool)
    r = np.repeat(np.arange(C["rows"]), np.diff(C["row_ptr"]))
    P[r, np.asarray(C["col_idx"], np.int64)] = True
    return P


def check_csr_invariants(C: dict):
    rp = np.asarray(C["row_ptr"], np.int64)
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == C["nnz"] == len(C["col_idx"])
    col = np.asarray(C["col_idx"], np.int64)
    for r in range(C["rows"]):
        seg = col[rp[r]:rp[r + 1]]
        assert np.all(np.diff(seg) > 0), f"row {r} not strictly ascending"
        assert seg.size == 0 or (seg[0] >= 0 and seg[-1] < C["cols"])


def check_dense_product(impl, A: synth.CSR, B: synth.CSR):
    """Integer-valued inputs: every sum is exact, so C must equal the dense product exactly,
    and C's pattern must equal the boolean product of the structural patterns."""
    C = impl(A, B)
    check_csr_invariants(C)
    Dexp = A.to_dense() @ B.to_dense()
    assert np.array_equal(dense_of(C), Dexp), "values differ from the dense product"
    Pexp = (A.pattern_dense().astype(np.int64) @ B.pattern_dense().astype(np.int64)) > 0
    assert np.array_equal(pattern_of(C), Pexp), "pattern differs from the structural product"


def laplacian_square_closed_form(n: int) -> dict:
    """(A^2) for A = 5-point Laplacian (4, -1) on an n x n grid, by grid geometry:
    diagonal 16 + (number of grid neighbours), -8 at distance 1, 2 on the grid
    diagonals, 1 at distance 2 along a grid line (every such pair has exactly
    these connecting paths inside the square)."""
    offs = [(-2, 0, 1.0), (-1, -1, 2.0), (-1, 0, -8.0), (-1, 1, 2.0), (0, -2, 1.0), (0, -1, -8.0),
            (0, 0, None), (0, 1, -8.0), (0, 2, 1.0), (1, -1, 2.0), (1, 0, -8.0), (1, 1, 2.0), (2, 0, 1.0)]
    rows, cols, vals = [], [], []
    rp = [0]
    for i in range(n):
        for j in range(n):
            deg = (i > 0) + (i < n - 1) + (j > 0) + (j < n - 1)
            for di, dj, v in offs:
                ii, jj = i + di, j + dj
                if 0 <= ii < n and 0 <= jj < n:
                    cols.append(ii * n + jj)
                    vals.append(16.0 + deg if v is None else v)
            rp.append(len(cols))
    return dict(rows=n * n, cols=n * n, row_ptr=np.array(rp, np.int64), col_idx=np.array(cols, np.int64),
                val=np.array(vals), nnz=len(cols))


def check_laplacian_square(impl, n: int):
    A = synth.laplacian5(n)
    C = impl(A, A)
    E = laplacian_square_closed_form(n)
    check_csr_invariants(C)
    assert np.array_equal(np.asarray(C["row_ptr"], np.int64), E["row_ptr"]), "row_ptr differs from closed form"
    assert np.array_equal(np.asarray(C["col_idx"], np.int64), E["col_idx"]), "col_idx differs from closed form"
    assert np.array_equal(np.asarray(C["val"]), E["val"]), "values differ from closed form"
    if n >= 2:
        assert C["nnz"] == 13 * n * n - 20 * n + 4
        assert C["F"] == 25 * (n - 2) ** 2 + 64 * (n - 2) + 36


def check_cancellation(impl):
    """A = [[1, 1]], B = [[1], [-1]]: the two products cancel, the entry is still stored."""
    A = synth.CSR(1, 2, np.array([0, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, 1.0]))
    B = synth.CSR(2, 1, np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([1.0, -1.0]))
    C = impl(A, B)
    assert C["nnz"] == 1 and list(C["col_idx"]) == [0] and C["val"][0] == 0.0
