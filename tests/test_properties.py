"""Property tests on random small inputs (hypothesis; skipped where it is not installed).

The oracle against the dense product and the boolean product of the structures, on integer
values (every sum exact) with empty rows, duplicate entries in a row, unsorted rows and explicit
zeros; the Combined CPU kernel against the oracle bit for bit on one thread and on several; and
the split of independent units among ranks."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import baseline  # noqa: E402
import oracle  # noqa: E402
from paper_1303_1651_gb300 import ranks, synth  # noqa: E402
from tests import pins  # noqa: E402


@st.composite
def csr(draw, rows=None, cols=None, max_dim=9, max_row=6):
    m = draw(st.integers(0, max_dim)) if rows is None else rows
    n = draw(st.integers(1, max_dim)) if cols is None else cols
    lens = [draw(st.integers(0, max_row)) for _ in range(m)]
    col = [draw(st.integers(0, n - 1)) for _ in range(sum(lens))]       # repeats and any order allowed
    val = [float(draw(st.integers(-3, 3))) for _ in range(sum(lens))]   # zeros included
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    return synth.CSR(m, n, rp, np.array(col, np.int32), np.array(val, np.float64))


@st.composite
def pair(draw):
    A = draw(csr())
    B = draw(csr(rows=A.cols))
    return A, B


@settings(max_examples=150, deadline=None)
@given(pair())
def test_oracle_equals_dense_and_boolean_products(ab):
    A, B = ab
    C = oracle.spgemm(A, B)
    pins.check_csr_invariants(C)
    assert np.array_equal(pins.dense_of(C), A.to_dense() @ B.to_dense())
    P = (A.pattern_dense().astype(np.int64) @ B.pattern_dense().astype(np.int64)) > 0
    assert np.array_equal(pins.pattern_of(C), P)
    assert C["F"] == int(np.diff(B.row_ptr)[A.col_idx.astype(np.int64)].sum()) if A.nnz else C["F"] == 0


@settings(max_examples=150, deadline=None)
@given(pair(), st.sampled_from([1, 2, 5]))
def test_combined_equals_oracle(ab, threads):
    A, B = ab
    R = oracle.spgemm(A, B)
    C = baseline.combined(A, B, threads)
    assert np.array_equal(C["row_ptr"], R["row_ptr"])
    assert np.array_equal(C["col_idx"].astype(np.int64), R["col_idx"])
    assert np.array_equal(C["val"].view(np.int64), R["val"].view(np.int64))


@given(st.integers(0, 10_000), st.integers(1, 64))
def test_shard_range_partitions(n, world):
    blocks = [ranks.shard_range(n, r, world) for r in range(world)]
    assert [i for b in blocks for i in b] == list(range(n))
    sizes = [len(b) for b in blocks]
    assert max(sizes) - min(sizes) <= 1
