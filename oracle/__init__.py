"""CPU oracle for C = A*B on CSR matrices (plain C, loaded through ctypes).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (no headers, helpers or tables) and imports nothing from
it.  The arithmetic lives in ``spgemm_oracle.c``; this file only marshals
numpy arrays and builds the shared object with gcc when it is missing.

Functions (each cites the passage of the paper it follows):
  spgemm(A, B)        -- Section IV-A row-major (Gustavson) algorithm with the
                         Section IV-B "Sort" store and a flag vector, keeping
                         structural zeros.  Returns pattern, values, the
                         per-entry sum of |a*b| (error scale), per-row
                         multiplication counts u and their total F.
  flops(A, B)         -- Section III multiplication count.
  grad(A, B, C, W)    -- gradients of sum(W * C) w.r.t. A's and B's values.
  transpose(A)        -- CSR -> CSC counting sort (Section IV-A conversion).
  batched(problems)   -- the plain oracle run once per independent problem.

Inputs are any objects with ``rows, cols, row_ptr, col_idx, val``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spgemm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_F64P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile spgemm_oracle.c into _build/liboracle.so (no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64 = ctypes.c_int64
            lib.oracle_flops.restype = i64
            lib.oracle_flops.argtypes = [i64, i64, _I64P, _I64P, _I64P]
            lib.oracle_spgemm.restype = i64
            lib.oracle_spgemm.argtypes = [i64, i64, i64, _I64P, _I64P, _F64P, _I64P, _I64P, _F64P,
                                          i64, _I64P, _I64P, _F64P, _F64P, _I64P, _I64P]
            lib.oracle_grad.restype = ctypes.c_int
            lib.oracle_grad.argtypes = [i64, i64, i64, _I64P, _I64P, _F64P, _I64P, _I64P, _F64P,
                                        _I64P, _I64P, _F64P, _F64P, _F64P]
            lib.oracle_transpose.restype = ctypes.c_int
            lib.oracle_transpose.argtypes = [i64, i64, _I64P, _I64P, _F64P, _I64P, _I64P, _F64P]
            _lib = lib
    return _lib


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int64)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def _check(A, B):
    if A.cols != B.rows:
        raise ValueError(f"inner dimensions differ: A is {A.rows}x{A.cols}, B is {B.rows}x{B.cols}")


def flops(A, B) -> int:
    """Number of multiplications: sum_k (nnz of column k of A) * (nnz of row k of B)."""
    _check(A, B)
    lib = _load()
    return int(lib.oracle_flops(A.rows, A.cols, _i64(A.row_ptr), _i64(A.col_idx), _i64(B.row_ptr)))


def spgemm(A, B) -> dict:
    """C = A*B.  Returns dict(row_ptr, col_idx, val, absval, count, u, F, nnz, rows, cols), int64 indices.

    absval is the sum of |a*b| of each entry (the scale of its rounding error), count the
    number of products in it."""
    _check(A, B)
    lib = _load()
    Arp, Acol, Aval = _i64(A.row_ptr), _i64(A.col_idx), _f64(A.val)
    Brp, Bcol, Bval = _i64(B.row_ptr), _i64(B.col_idx), _f64(B.val)
    F = int(lib.oracle_flops(A.rows, A.cols, Arp, Acol, Brp)) if A.rows else 0
    cap = max(F, 1)
    Crp = np.zeros(A.rows + 1, np.int64)
    Ccol = np.empty(cap, np.int64)
    Cval = np.empty(cap, np.float64)
    Cabs = np.empty(cap, np.float64)
    Ccnt = np.empty(cap, np.int64)
    u = np.zeros(max(A.rows, 1), np.int64)
    nnz = int(lib.oracle_spgemm(A.rows, A.cols, B.cols, Arp, Acol, Aval, Brp, Bcol, Bval,
                                cap, Crp, Ccol, Cval, Cabs, Ccnt, u))
    if nnz < 0:
        raise RuntimeError(f"oracle_spgemm failed ({nnz})")
    return dict(rows=A.rows, cols=B.cols, row_ptr=Crp, col_idx=Ccol[:nnz].copy(),
                val=Cval[:nnz].copy(), absval=Cabs[:nnz].copy(), count=Ccnt[:nnz].copy(), u=u[:A.rows].copy(),
                F=F, nnz=nnz)


def grad(A, B, C: dict, W) -> tuple[np.ndarray, np.ndarray]:
    """(dA, dB) of loss = sum over C's entries of W*C; W aligned with C's entries."""
    _check(A, B)
    lib = _load()
    dA = np.zeros(max(int(A.row_ptr[-1]) if A.rows else 0, 1), np.float64)
    dB = np.zeros(max(int(B.row_ptr[-1]) if B.rows else 0, 1), np.float64)
    rc = lib.oracle_grad(A.rows, A.cols, B.cols, _i64(A.row_ptr), _i64(A.col_idx), _f64(A.val),
                         _i64(B.row_ptr), _i64(B.col_idx), _f64(B.val),
                         _i64(C["row_ptr"]), _i64(C["col_idx"]), _f64(W), dA, dB)
    if rc != 0:
        raise RuntimeError(f"oracle_grad failed ({rc})")
    nA = int(A.row_ptr[-1]) if A.rows else 0
    nB = int(B.row_ptr[-1]) if B.rows else 0
    return dA[:nA].copy(), dB[:nB].copy()


def transpose(A) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """CSC of A: (col_ptr[n+1], row_idx[nnz], val[nnz]), rows ascending within a column."""
    lib = _load()
    nnz = int(A.row_ptr[-1]) if A.rows else 0
    cp = np.zeros(A.cols + 1, np.int64)
    ri = np.zeros(max(nnz, 1), np.int64)
    tv = np.zeros(max(nnz, 1), np.float64)
    rc = lib.oracle_transpose(A.rows, A.cols, _i64(A.row_ptr), _i64(A.col_idx), _f64(A.val), cp, ri, tv)
    if rc != 0:
        raise RuntimeError("oracle_transpose failed")
    return cp, ri[:nnz].copy(), tv[:nnz].copy()


def batched(problems) -> list[dict]:
    """The plain oracle applied to each independent (A, B) problem in turn."""
    return [spgemm(A, B) for A, B in problems]
