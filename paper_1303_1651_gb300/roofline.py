"""Traffic and flop accounting for C = A*B, and the paper's balance model.

Flops (Section III): two per multiplication, the worst-case convention, where
the multiplications are F = sum_k nnz(A(:,k)) * nnz(B(k,:)) = sum_r u_r.

Minimal traffic of the product (what any implementation must move through
HBM once): read A (row pointer and the index and value of each entry), read
each row of B that A references once, write C.  With int32 indices and
float64 values an entry is 12 bytes and a row pointer 4 bytes:

    bytes_min = 4(m+1) + 12 nnz(A) + 4 k_ref + 12 sum_{j referenced} nnz(B_j)
                + 4(m+1) + 12 nnz(C)

where k_ref counts the referenced rows of B (two row-pointer reads each,
mostly shared with the neighbouring row, counted as one).

The paper's light-speed model (Section IV-A) is P = min(P_max, b_max / B_c)
(printed with max; the roofline is the minimum), with the inner loop of the
row-major kernel moving an 8-byte index, an 8-byte value and loading and
storing one 8-byte temporary per two flops: B_c = 16 bytes/flop.
"""
from __future__ import annotations

import numpy as np

IDX_BYTES = 4
VAL_BYTES = 8


def products_per_row(A, B) -> np.ndarray:
    blen = np.diff(np.asarray(B.row_ptr, np.int64))
    contrib = blen[np.asarray(A.col_idx, np.int64)]
    rows = np.repeat(np.arange(A.rows), np.diff(np.asarray(A.row_ptr, np.int64)))
    return np.bincount(rows, weights=contrib, minlength=A.rows).astype(np.int64)


def flops(F: int) -> int:
    return 2 * int(F)


def bytes_min(A, B, nnz_c: int) -> int:
    m = A.rows
    ref = np.zeros(B.rows, bool)
    ref[np.asarray(A.col_idx, np.int64)] = True
    blen = np.diff(np.asarray(B.row_ptr, np.int64))
    b_bytes = IDX_BYTES * int(ref.sum()) + (IDX_BYTES + VAL_BYTES) * int(blen[ref].sum())
    a_bytes = IDX_BYTES * (m + 1) + (IDX_BYTES + VAL_BYTES) * int(A.row_ptr[-1] if m else 0)
    c_bytes = IDX_BYTES * (m + 1) + (IDX_BYTES + VAL_BYTES) * int(nnz_c)
    return a_bytes + b_bytes + c_bytes


def code_balance_gustavson(idx_bytes: int = 8, val_bytes: int = 8) -> float:
    """Bytes per flop of the row-major inner loop: load index, load value, load+store temp; 2 flops."""
    return (idx_bytes + val_bytes + 2 * val_bytes) / 2.0


def light_speed(p_max: float, bandwidth: float, balance: float) -> float:
    """Roofline P = min(P_max, b_max / B_c)."""
    return min(p_max, bandwidth / balance)


def l1_limit_flops(clock_hz: float, loads_per_cycle: float = 2.0, ldst_per_iter: tuple = (3, 1)) -> float:
    """In-L1 limit of the inner loop: 3 loads + 1 store per 2 flops, with 2 loads or 1 load + 1 store
    per cycle -> 2 cycles per iteration -> 1 flop per cycle."""
    loads, stores = ldst_per_iter
    cycles = max(stores + (loads - stores) / loads_per_cycle, (loads + stores) / loads_per_cycle)
    return 2.0 * clock_hz / cycles
