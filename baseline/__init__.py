"""The paper's "Combined" CSR x CSR kernel (Section IV-B) on the host cores: a second, optimised
CPU baseline beside the plain oracle.

Not the oracle and not on the GPU path.  ``bench.py`` times it (``cpu_baseline_combined``) and
``tests/test_combined_baseline.py`` checks it against the oracle.  The arithmetic lives in
``combined.cpp``; this file builds it with the host C++ compiler (with OpenMP when the compiler
has it) and marshals numpy arrays.

  combined(A, B, threads=None) -> dict(rows, cols, row_ptr, col_idx, val, nnz, F, rows_minmax,
                                       rows_sort, threads)

Inputs are any objects with ``rows, cols, row_ptr, col_idx, val`` (int32 indices are used as
they are; other integer types are converted).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "combined.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libcombined.so")
_lock = threading.Lock()
_lib = None

_I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_F64P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile combined.cpp into _build/libcombined.so: -O3, no FMA contraction, OpenMP if available."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        base = ["c++", "-O3", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except (subprocess.CalledProcessError, OSError):
            subprocess.check_call(base)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64 = ctypes.c_int64
            lib.combined_max_threads.restype = ctypes.c_int
            lib.combined_max_threads.argtypes = []
            lib.combined_products.restype = i64
            lib.combined_products.argtypes = [i64, i64, _I32P, _I32P, _I32P, _I64P]
            lib.combined_spgemm.restype = i64
            lib.combined_spgemm.argtypes = [i64, i64, i64, _I32P, _I32P, _F64P, _I32P, _I32P, _F64P, _I64P, i64,
                                            ctypes.c_int, _I64P, _I32P, _F64P, _I32P, _F64P, _I64P]
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().combined_max_threads())


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def combined(A, B, threads: int | None = None) -> dict:
    """C = A * B by the Combined kernel; threads defaults to every thread OpenMP offers."""
    if A.cols != B.rows:
        raise ValueError(f"inner dimensions differ: A is {A.rows}x{A.cols}, B is {B.rows}x{B.cols}")
    lib = _load()
    threads = max_threads() if threads is None else max(1, int(threads))
    Arp, Acol, Aval = _i32(A.row_ptr), _i32(A.col_idx), _f64(A.val)
    Brp, Bcol, Bval = _i32(B.row_ptr), _i32(B.col_idx), _f64(B.val)
    u = np.empty(max(A.rows, 1), np.int64)
    F = int(lib.combined_products(A.rows, A.cols, Arp, Acol, Brp, u))
    if F < 0:
        raise ValueError("a column index of A is out of range")
    cap = max(F, 1)
    C_rp = np.empty(A.rows + 1, np.int64)
    C_col = np.empty(cap, np.int32)
    C_val = np.empty(cap, np.float64)
    one = threads <= 1
    S_col = C_col[:1] if one else np.empty(cap, np.int32)
    S_val = C_val[:1] if one else np.empty(cap, np.float64)
    stats = np.zeros(2, np.int64)
    nnz = int(lib.combined_spgemm(A.rows, A.cols, B.cols, Arp, Acol, Aval, Brp, Bcol, Bval, u, F, threads,
                                  C_rp, C_col, C_val, S_col, S_val, stats))
    if nnz == -1:
        raise ValueError("a column index of B is out of range")
    if nnz == -2:
        raise MemoryError("combined_spgemm could not allocate its temporary vectors")
    if nnz < 0:
        raise RuntimeError(f"combined_spgemm failed ({nnz})")
    return dict(rows=A.rows, cols=B.cols, row_ptr=C_rp, col_idx=C_col[:nnz], val=C_val[:nnz], nnz=nnz, F=F,
                rows_minmax=int(stats[0]), rows_sort=int(stats[1]), threads=threads)
