"""Seeded synthetic CSR inputs shaped like the paper's two test structures.

This module only builds inputs; it holds none of the product's arithmetic, so
both the CUDA path and the CPU oracle can be fed from it.

Structures (Section III of the paper, "Benchmark Platform and Test-Cases"):

* ``laplacian5(n)`` -- the five-band matrix of a 5-point finite-difference
  stencil for a Dirichlet problem on an n x n square grid.  The paper does not
  print the stencil values; we use 4 on the diagonal and -1 for every existing
  grid neighbour, grid index r = i*n + j, no coupling across the ends of grid
  rows.  nnz = 5n^2 - 4n.
* ``random_k(N, k, seed)`` -- a square matrix with exactly k distinct,
  uniformly placed columns per row (the paper uses 5 per row), values U(-1, 1).
* ``random_fill(N, fill, seed)`` -- the same generator with a fixed fill ratio
  per row (the paper's 0.1 % fill experiment).
* ``batch_problems(count, seed)`` -- uneven independent problems for the
  batched form: N log-uniform in [256, 65536], half Laplacian^2, half
  random*random with k ~ U{2..32}.

Rows come out sorted by column with no duplicates, unless a helper below
deliberately breaks that (``shuffle_rows``, ``duplicate_entries``).
Random streams are numpy's Philox counter-based generator, seeded explicitly.
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np

SEED_A = 1303
SEED_B = 1651
SEED_W = 42
SEED_BATCH = 2026


@dataclass
class CSR:
    """Host CSR matrix: int32 row_ptr (rows+1), int32 col_idx (nnz), float64 val (nnz)."""

    rows: int
    cols: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if self.rows > 0 else 0

    def copy(self) -> "CSR":
        return CSR(self.rows, self.cols, self.row_ptr.copy(), self.col_idx.copy(), self.val.copy())

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.rows, self.cols), dtype=np.float64)
        r = np.repeat(np.arange(self.rows), np.diff(self.row_ptr))
        np.add.at(d, (r, self.col_idx.astype(np.int64)), self.val)
        return d

    def pattern_dense(self) -> np.ndarray:
        d = np.zeros((self.rows, self.cols), dtype=bool)
        r = np.repeat(np.arange(self.rows), np.diff(self.row_ptr))
        d[r, self.col_idx.astype(np.int64)] = True
        return d


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def _from_rows(rows: int, cols: int, counts: np.ndarray, col_idx: np.ndarray, val: np.ndarray) -> CSR:
    row_ptr = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise OverflowError("nnz exceeds int32 CSR")
    return CSR(rows, cols, row_ptr.astype(np.int32), col_idx.astype(np.int32, copy=False),
               np.ascontiguousarray(val, dtype=np.float64))


def laplacian5(n: int, diag: float = 4.0, off: float = -1.0) -> CSR:
    """5-point stencil on an n x n grid, Dirichlet boundary, row r = i*n + j."""
    if n <= 0:
        return CSR(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    N = n * n
    r = np.arange(N, dtype=np.int64)
    i, j = r // n, r % n
    # neighbours in ascending column order: up (r-n), left (r-1), self, right (r+1), down (r+n)
    cand = np.stack([r - n, r - 1, r, r + 1, r + n], axis=1)
    ok = np.stack([i > 0, j > 0, np.ones(N, bool), j < n - 1, i < n - 1], axis=1)
    vals = np.broadcast_to(np.array([off, off, diag, off, off]), (N, 5))
    counts = ok.sum(axis=1)
    return _from_rows(N, N, counts, cand[ok], vals[ok])


def _distinct_sorted_cols(rng: np.random.Generator, nrows: int, k: int, ncols: int) -> np.ndarray:
    """nrows x k array, each row k distinct columns drawn uniformly from [0, ncols), ascending."""
    if k > ncols:
        raise ValueError("k distinct columns need k <= ncols")
    out = np.empty((nrows, k), dtype=np.int64)
    chunk = 1 << 20
    for s in range(0, nrows, chunk):
        e = min(nrows, s + chunk)
        c = rng.integers(0, ncols, size=(e - s, k), dtype=np.int64)
        c.sort(axis=1)
        bad = np.nonzero((c[:, 1:] == c[:, :-1]).any(axis=1))[0] if k > 1 else np.zeros(0, np.int64)
        while bad.size:
            redo = rng.integers(0, ncols, size=(bad.size, k), dtype=np.int64)
            redo.sort(axis=1)
            c[bad] = redo
            still = (redo[:, 1:] == redo[:, :-1]).any(axis=1)
            bad = bad[still]
        out[s:e] = c
    return out


def random_k(N: int, k: int, seed: int, ncols: int | None = None) -> CSR:
    """N x ncols matrix, exactly k distinct uniform columns per row, values U(-1, 1)."""
    ncols = N if ncols is None else ncols
    rng = _rng(seed)
    cols = _distinct_sorted_cols(rng, N, k, ncols).reshape(-1)
    val = rng.uniform(-1.0, 1.0, size=N * k)
    return _from_rows(N, ncols, np.full(N, k, np.int64), cols, val)


def random_lengths(lengths: np.ndarray, ncols: int, seed: int) -> CSR:
    """Rows with up to lengths[r] distinct uniform columns (draws that collide are merged), U(-1,1)."""
    rng = _rng(seed)
    lengths = np.asarray(lengths, dtype=np.int64)
    m = lengths.size
    rows = np.repeat(np.arange(m, dtype=np.int64), lengths)
    cols = rng.integers(0, max(ncols, 1), size=rows.size, dtype=np.int64)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    keep = np.ones(rows.size, bool)
    if rows.size:
        keep[1:] = (rows[1:] != rows[:-1]) | (cols[1:] != cols[:-1])
    rows, cols = rows[keep], cols[keep]
    counts = np.bincount(rows, minlength=m)
    val = rng.uniform(-1.0, 1.0, size=cols.size)
    return _from_rows(m, ncols, counts, cols, val)


def random_fill(N: int, fill: float, seed: int) -> CSR:
    """Square random matrix with max(1, round(fill*N)) distinct columns per row."""
    k = max(1, int(round(fill * N)))
    return random_k(N, k, seed)


def power_law(m: int, ncols: int, seed: int, alpha: float = 1.6, max_len: int | None = None) -> CSR:
    """Row lengths ~ Zipf(alpha) clipped to max_len: a skewed degree distribution."""
    rng = _rng(seed + 7)
    max_len = ncols if max_len is None else min(max_len, ncols)
    lengths = np.minimum(rng.zipf(alpha, size=m), max_len)
    return random_lengths(lengths, ncols, seed)


def sweep_sizes() -> list[int]:
    """13 log-spaced N from 1e3 to 1e7: round(10^(3 + i/3))."""
    return [int(round(10 ** (3 + i / 3))) for i in range(13)]


SWEEP_KINDS = ("lap", "rand4", "rand8", "rand16")


def sweep_points() -> list[tuple[int, str]]:
    """Every (N, kind) of the size sweep, in increasing N."""
    return [(N, kind) for N in sweep_sizes() for kind in SWEEP_KINDS]


def sweep_problem(N: int, kind: str) -> tuple[CSR, CSR]:
    """One point of the size sweep.  'lap': C = A*A with A the 5-point Laplacian on a
    round(sqrt(N))^2 grid (B is A).  'rand<k>': A and B are N x N with k distinct uniform columns
    per row, seeds SEED_A + N and SEED_B + N."""
    if kind == "lap":
        A = laplacian5(max(2, int(round(math.sqrt(N)))))
        return A, A
    if not kind.startswith("rand"):
        raise ValueError(f"unknown sweep kind {kind!r}")
    k = int(kind[4:])
    return random_k(N, k, SEED_A + N), random_k(N, k, SEED_B + N)


def batch_problems(count: int = 512, seed: int = SEED_BATCH, nmin: int = 256, nmax: int = 65536):
    """Independent (A, B) pairs of uneven sizes: first half Laplacian^2 (B is A), second half random*random."""
    rng = _rng(seed)
    logs = rng.uniform(math.log(nmin), math.log(nmax), size=count)
    sizes = np.rint(np.exp(logs)).astype(np.int64)
    ks = rng.integers(2, 33, size=count)
    probs = []
    for t in range(count):
        if t < count // 2:
            n = max(2, int(round(math.sqrt(sizes[t]))))
            A = laplacian5(n)
            probs.append((A, A))
        else:
            N, k = int(sizes[t]), int(ks[t])
            A = random_k(N, k, seed + 2 * t + 1)
            B = random_k(N, k, seed + 2 * t + 2)
            probs.append((A, B))
    return probs


def shuffle_rows(A: CSR, seed: int) -> CSR:
    """Same matrix with the entries of every row in a random order."""
    rng = _rng(seed)
    out = A.copy()
    r = np.repeat(np.arange(A.rows, dtype=np.int64), np.diff(A.row_ptr))
    order = np.lexsort((rng.random(A.nnz), r))
    out.col_idx = A.col_idx[order].copy()
    out.val = A.val[order].copy()
    return out


def duplicate_entries(A: CSR, seed: int, frac: float = 0.2) -> CSR:
    """Append a copy of a random fraction of each row's entries (new values) to the row, unsorted."""
    rng = _rng(seed)
    r = np.repeat(np.arange(A.rows, dtype=np.int64), np.diff(A.row_ptr))
    pick = rng.random(A.nnz) < frac
    rows = np.concatenate([r, r[pick]])
    cols = np.concatenate([A.col_idx.astype(np.int64), A.col_idx[pick].astype(np.int64)])
    vals = np.concatenate([A.val, rng.uniform(-1, 1, size=int(pick.sum()))])
    order = np.lexsort((rng.random(rows.size), rows))
    counts = np.bincount(rows, minlength=A.rows)
    return _from_rows(A.rows, A.cols, counts, cols[order], vals[order])


def integer_valued(A: CSR, seed: int, lo: int = -3, hi: int = 3) -> CSR:
    """Same pattern with nonzero integer values in [lo, hi] (sums of products are then exact)."""
    rng = _rng(seed)
    v = rng.integers(lo, hi, size=A.nnz, endpoint=True).astype(np.float64)
    v[v == 0] = 1.0
    out = A.copy()
    out.val = v
    return out


def from_dense(D: np.ndarray, keep_zeros_mask: np.ndarray | None = None) -> CSR:
    """CSR of a dense array; entries where D != 0 (or where keep_zeros_mask is set) are structural."""
    D = np.asarray(D, dtype=np.float64)
    mask = D != 0 if keep_zeros_mask is None else (keep_zeros_mask | (D != 0))
    r, c = np.nonzero(mask)
    counts = np.bincount(r, minlength=D.shape[0])
    return _from_rows(D.shape[0], D.shape[1], counts, c, D[r, c])
