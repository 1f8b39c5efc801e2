"""The C-ABI library builds, loads and exports every entry point declared in include/*.h.
Host-only argument checks run without a GPU (no kernel is launched)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1303_1651_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(spgemm_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_every_declared_symbol_exported(lib):
    names = declared_functions()
    assert "spgemm_plan" in names and "spgemm_numeric" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_error_strings(lib):
    for code in range(11):
        s = binding.error_string(code)
        assert isinstance(s, str) and s
    assert binding.error_string(12345) == "unknown status"


def _desc(rows, cols, nnz=0):
    return binding.spgemm_csr_t(rows, cols, nnz, 0x1000 if rows > 0 else None, 0x2000 if nnz else None, None)


def test_workspace_size_host_only(lib):
    A, B = _desc(1000, 500, 10), _desc(500, 700, 10)
    n = ctypes.c_size_t(0)
    assert lib.spgemm_workspace_size(ctypes.byref(A), ctypes.byref(B), None, ctypes.byref(n)) == 0
    # grows with rows of A and columns of B (dense accumulator slabs)
    A2 = _desc(2000, 500, 10)
    n2 = ctypes.c_size_t(0)
    assert lib.spgemm_workspace_size(ctypes.byref(A2), ctypes.byref(B), None, ctypes.byref(n2)) == 0
    assert n2.value > n.value
    opt = binding.options(dense_slabs=8)
    n3 = ctypes.c_size_t(0)
    assert lib.spgemm_workspace_size(ctypes.byref(A), ctypes.byref(B), ctypes.byref(opt), ctypes.byref(n3)) == 0
    assert n3.value > n.value


def test_invalid_arguments_rejected_on_host(lib):
    A, B = _desc(10, 5, 3), _desc(6, 7, 3)      # inner dimensions differ
    n = ctypes.c_size_t(0)
    assert lib.spgemm_workspace_size(ctypes.byref(A), ctypes.byref(B), None, ctypes.byref(n)) == 1
    h = ctypes.c_void_p(0)
    B2 = _desc(5, 7, 3)
    # NULL workspace -> INVALID before any device work
    assert lib.spgemm_plan(ctypes.byref(h), ctypes.byref(A), ctypes.byref(B2), None, None, 0, None) == 1
    # misaligned workspace -> INVALID
    assert lib.spgemm_plan(ctypes.byref(h), ctypes.byref(A), ctypes.byref(B2), None, 0x1001, 1 << 30, None) == 1
    # too small workspace -> ALLOC
    assert lib.spgemm_plan(ctypes.byref(h), ctypes.byref(A), ctypes.byref(B2), None, 0x100000, 16, None) == 2
    neg = _desc(-1, 5)
    assert lib.spgemm_workspace_size(ctypes.byref(neg), ctypes.byref(B2), None, ctypes.byref(n)) == 1
    # calls out of order on a NULL plan
    assert lib.spgemm_symbolic(None, 0x1000, ctypes.byref(ctypes.c_int64()), None) == 7
    assert lib.spgemm_numeric(None, None, None, None, None, None) == 7
    assert lib.spgemm_free(None) == 0
    # pattern reuse needs a plan (and a recorded map)
    assert lib.spgemm_replay_size(None, ctypes.byref(ctypes.c_size_t())) == 7
    assert lib.spgemm_replay_record(None, None, 0x1000, 1 << 20, None) == 7
    assert lib.spgemm_replay(None, None, None, 0x1000, None, None, None) == 7
    # the no-workspace scan checks its arguments and its size limit before any CUDA call
    total = ctypes.c_int64(-1)
    assert lib.spgemm_scan_counts_noalloc(None, 10, ctypes.byref(total), None) == 1
    assert lib.spgemm_scan_counts_noalloc(0x1000, -1, ctypes.byref(total), None) == 1
    assert lib.spgemm_scan_counts_noalloc(0x1000, (1 << 26), ctypes.byref(total), None) == 10
    assert total.value == -1


def test_struct_sizes_match_header(lib):
    # spgemm_options_t: 16 int32; spgemm_csr_t: 2 int32 + int64 + 3 pointers
    assert ctypes.sizeof(binding.spgemm_options_t) == 64
    assert ctypes.sizeof(binding.spgemm_csr_t) == 40
    assert ctypes.sizeof(binding.spgemm_info_t) == 40


def test_options_fields_follow_the_header():
    # the ctypes mirror lists spgemm_options_t's fields in the header's order
    text = open(os.path.join(ROOT, "include", "spgemm_gb300.h")).read()
    body = text[text.index("typedef struct {\n  int32_t merge_max_k;"):]
    body = body[:body.index("} spgemm_options_t;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"int32_t\s+([a-z0-9_]+)", body)
    assert names == [f[0] for f in binding.spgemm_options_t._fields_]


def test_storage_options_checked_on_host(lib):
    A, B = _desc(1000, 500, 10), _desc(500, 700, 10)
    plain, csc = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert lib.spgemm_workspace_size(ctypes.byref(A), ctypes.byref(B), None, ctypes.byref(plain)) == 0
    opt = binding.options(a_storage=1, b_storage=1)
    assert lib.spgemm_workspace_size(ctypes.byref(A), ctypes.byref(B), ctypes.byref(opt), ctypes.byref(csc)) == 0
    assert csc.value > plain.value           # the converted structures, values and gradients
    bad = binding.options(b_storage=2)
    assert lib.spgemm_workspace_size(ctypes.byref(A), ctypes.byref(B), ctypes.byref(bad), ctypes.byref(csc)) == 1
    # a descriptor given by columns needs its column pointers
    A_cols = binding.spgemm_csr_t(0, 500, 0, None, None, None)
    assert lib.spgemm_workspace_size(ctypes.byref(A_cols), ctypes.byref(B), ctypes.byref(opt), ctypes.byref(csc)) == 1


def test_fault_injection_alloc_on_host(lib, monkeypatch):
    A, B = _desc(10, 5, 3), _desc(5, 7, 3)
    h = ctypes.c_void_p(0)
    monkeypatch.setenv("SPGEMM_FAULT", "alloc")
    assert lib.spgemm_plan(ctypes.byref(h), ctypes.byref(A), ctypes.byref(B), None, 0x100000, 1 << 40, None) == 2
