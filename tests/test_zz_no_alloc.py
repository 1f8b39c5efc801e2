"""spgemm_scan_counts_noalloc, the scan entry point that takes no workspace, called through the
C ABI and checked against spgemm_symbolic, the entry point that builds C's row pointers with a
caller workspace: the per-row counts of C go in, and the same row pointers and nnz(C) must come
out, bit for bit, on consecutive calls that share the library's one fixed scratch array.

This file is collected last so that it also runs after the rest of the GPU suite in one process."""
import ctypes

import pytest
import torch

from paper_1303_1651_gb300 import binding, synth

pytestmark = pytest.mark.gpu

MAX_ROWS = (1 << 26) - 1          # SPGEMM_NOALLOC_MAX_ROWS
ST_OVERFLOW, ST_SCRATCH_LIMIT = 3, 10


def _symbolic_row_ptr(A, B):
    """C's row pointers and nnz(C) from the workspace path (spgemm_plan + spgemm_symbolic)."""
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    ws = torch.empty(binding.spgemm_workspace_size(dA, dB), dtype=torch.uint8, device="cuda")
    plan = binding.spgemm_plan(dA, dB, ws)
    try:
        rp = torch.empty(A.rows + 1, dtype=torch.int32, device="cuda")
        nnz = binding.spgemm_symbolic(plan, rp)
    finally:
        binding.spgemm_free(plan)
    return rp, nnz


def _counts_buffer(rp):
    """rows + 1 entries: the per-row counts, then a value the scan must ignore."""
    buf = torch.empty_like(rp)
    buf[:-1] = rp[1:] - rp[:-1]
    buf[-1] = -12345
    return buf


def _noalloc(buf, rows, stream=None):
    lib = binding.load()
    total = ctypes.c_int64(-1)
    s = stream if stream is not None else torch.cuda.current_stream()
    st = lib.spgemm_scan_counts_noalloc(ctypes.c_void_p(buf.data_ptr()), ctypes.c_int64(rows), ctypes.byref(total),
                                        ctypes.c_void_p(s.cuda_stream))
    return st, total.value


def test_matches_symbolic_on_consecutive_calls():
    # products whose row counts span many 2048-row scan tiles and end in a ragged tile
    products = [(synth.random_k(100_003, 8, seed=11), synth.random_k(100_003, 8, seed=12)),
                (synth.laplacian5(300), synth.laplacian5(300)),
                (synth.random_k(5_000, 3, seed=13), synth.random_k(5_000, 3, seed=14))]
    expected = [_symbolic_row_ptr(A, B) for A, B in products]
    for call in range(2):                     # the same sequence twice: scratch state must not leak
        for rp, nnz in expected:
            buf = _counts_buffer(rp)
            st, total = _noalloc(buf, rp.numel() - 1)
            assert st == 0, binding.error_string(st)
            assert total == nnz
            assert torch.equal(buf, rp), f"call round {call}: row pointers differ"


def test_empty_and_overflow():
    buf = torch.full((1,), 77, dtype=torch.int32, device="cuda")
    assert _noalloc(buf, 0) == (0, 0)
    assert int(buf[0]) == 0
    big = torch.tensor([1 << 30, 1 << 30, 1 << 30, 0], dtype=torch.int32, device="cuda")
    st, total = _noalloc(big, 3)
    assert st == ST_OVERFLOW and total == 3 << 30
    # the prefix sums that do not fit are stored as INT32_MAX
    assert big.tolist() == [0, 1 << 30, (1 << 31) - 1, (1 << 31) - 1]


def test_size_limit():
    # the largest accepted size: every count 1, so row_ptr[r] = r
    buf = torch.ones(MAX_ROWS + 2, dtype=torch.int32, device="cuda")
    st, total = _noalloc(buf, MAX_ROWS)
    assert st == 0 and total == MAX_ROWS
    assert torch.equal(buf[:MAX_ROWS + 1], torch.arange(MAX_ROWS + 1, dtype=torch.int32, device="cuda"))
    # one row more is refused before any device work (the buffer is large enough either way)
    buf.fill_(5)
    st, total = _noalloc(buf, MAX_ROWS + 1)
    assert st == ST_SCRATCH_LIMIT and total == -1
    torch.cuda.synchronize()
    assert int(buf.min()) == 5 and int(buf.max()) == 5
    with pytest.raises(binding.SpgemmError, match="SCRATCH_LIMIT"):
        binding.spgemm_scan_counts_noalloc(buf, MAX_ROWS + 1)


def test_ordered_on_a_caller_stream():
    # The counts are written by kernels queued on a side stream (behind a spin of about a
    # millisecond), and the entry point is called on that stream with no host synchronisation in
    # between: its clearing of the scratch, its scan and its read-back must run after them.
    A, B = synth.random_k(50_001, 6, seed=21), synth.random_k(50_001, 6, seed=22)
    rp, nnz = _symbolic_row_ptr(A, B)
    counts = rp[1:] - rp[:-1]
    buf = torch.full_like(rp, -1)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        torch.cuda._sleep(2_000_000)
        torch.add(counts, 0, out=buf[:-1])
        st, total = _noalloc(buf, rp.numel() - 1, stream=side)
    assert st == 0, binding.error_string(st)
    assert total == nnz
    torch.cuda.synchronize()
    assert torch.equal(buf, rp)
