"""Checks of the size sweep that hold at any size, shared by the GPU sweep test and its CPU
self-test: C's structure checked whole where it lies (device or host tensors), the Laplacian²
from its closed form, and the oracle's rows for a sample of rows of A."""
import numpy as np
import torch

from paper_1303_1651_gb300 import synth


def products_count(A, B) -> int:
    """F: the lengths of the rows of B, summed over the entries of A."""
    return int(np.diff(np.asarray(B.row_ptr, np.int64))[np.asarray(A.col_idx, np.int64)].sum())


def check_structure(C_rp, C_col, nnz, cols):
    """C's row pointer runs from 0 to nnz without decreasing; columns lie in [0, cols) and ascend
    strictly within every row.  Works on the tensors where they lie."""
    rp = C_rp.long()
    assert int(rp[0]) == 0 and int(rp[-1]) == nnz
    assert bool((rp[1:] >= rp[:-1]).all()), "row pointer decreases"
    if nnz == 0:
        return
    assert int(C_col.min()) >= 0 and int(C_col.max()) < cols, "column out of range"
    ascending = C_col[1:] > C_col[:-1]
    starts = rp[1:-1]
    starts = starts[(starts > 0) & (starts < nnz)]
    ascending[starts - 1] = True            # a row boundary lies between positions s - 1 and s
    assert bool(ascending.all()), "columns not strictly ascending within a row"


def laplacian_square(n: int, device="cuda"):
    """(A^2) for the 5-point Laplacian (4, -1) on an n x n grid, n >= 5, from its closed form, as
    tensors on the given device: row pointer, columns and values."""
    offs = [(-2, 0, 1.0), (-1, -1, 2.0), (-1, 0, -8.0), (-1, 1, 2.0), (0, -2, 1.0), (0, -1, -8.0), (0, 0, 0.0),
            (0, 1, -8.0), (0, 2, 1.0), (1, -1, 2.0), (1, 0, -8.0), (1, 1, 2.0), (2, 0, 1.0)]
    di = torch.tensor([o[0] for o in offs], device=device)
    dj = torch.tensor([o[1] for o in offs], device=device)
    r = torch.arange(n * n, device=device)
    i, j = r // n, r % n
    ii, jj = i[:, None] + di, j[:, None] + dj
    valid = (ii >= 0) & (ii < n) & (jj >= 0) & (jj < n)
    val = torch.tensor([o[2] for o in offs], dtype=torch.float64, device=device).repeat(n * n, 1)
    val[:, 6] = 16.0 + ((i > 0).double() + (i < n - 1).double() + (j > 0).double() + (j < n - 1).double())
    rp = torch.zeros(n * n + 1, dtype=torch.int64, device=device)
    rp[1:] = torch.cumsum(valid.sum(1), 0)
    return rp, (ii * n + jj)[valid], val[valid]


def sample_rows(m: int, seed: int, count: int = 512) -> np.ndarray:
    """The first and last 8 rows and a seeded sample, sorted, without repeats."""
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([np.arange(min(8, m)), np.arange(max(0, m - 8), m),
                                     rng.integers(0, m, count)])).astype(np.int64)


def ranges(starts, ends) -> np.ndarray:
    """The concatenation of arange(s, e) over the pairs."""
    lens = ends - starts
    return np.repeat(starts - np.cumsum(np.concatenate([[0], lens[:-1]])), lens) + np.arange(lens.sum())


def sub_problem(A, B, rows):
    """The given rows of A, and the rows of B they reference (renumbered): the same rows of C, with
    every product in the same loop order."""
    arp = np.asarray(A.row_ptr, np.int64)
    aidx = ranges(arp[rows], arp[rows + 1])
    ref, inv = np.unique(np.asarray(A.col_idx, np.int64)[aidx], return_inverse=True)
    brp = np.asarray(B.row_ptr, np.int64)
    bidx = ranges(brp[ref], brp[ref + 1])
    A_sub = synth.CSR(len(rows), len(ref), np.concatenate([[0], np.cumsum(arp[rows + 1] - arp[rows])]).astype(np.int32),
                      inv.astype(np.int32), np.asarray(A.val)[aidx])
    B_sub = synth.CSR(len(ref), B.cols, np.concatenate([[0], np.cumsum(brp[ref + 1] - brp[ref])]).astype(np.int32),
                      np.asarray(B.col_idx)[bidx], np.asarray(B.val)[bidx])
    return A_sub, B_sub


def gpu_rows(C_rp, C_col, C_val, rows, cols) -> dict:
    """The given rows of C (tensors on any device) as a host CSR dict."""
    rp = C_rp.cpu().numpy().astype(np.int64)
    idx = torch.from_numpy(ranges(rp[rows], rp[rows + 1])).to(C_col.device)
    lens = rp[rows + 1] - rp[rows]
    return dict(rows=len(rows), cols=cols, row_ptr=np.concatenate([[0], np.cumsum(lens)]),
                col_idx=C_col[idx].cpu().numpy(), val=C_val[idx].cpu().numpy())
