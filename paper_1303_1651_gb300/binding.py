"""ctypes binding of the C ABI in include/spgemm_gb300.h (argument marshalling only).

Every step of the product runs in the CUDA library; this module turns torch
tensors into device pointers and sizes, passes the current CUDA stream, and
raises ``SpgemmError`` on a non-zero status.  If the library has not been
built, ``load()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

_lib = None

SPGEMM_STATUS = {
    0: "SPGEMM_OK", 1: "SPGEMM_ERR_INVALID", 2: "SPGEMM_ERR_ALLOC", 3: "SPGEMM_ERR_OVERFLOW",
    4: "SPGEMM_ERR_TABLE_FULL", 5: "SPGEMM_ERR_CUDA", 6: "SPGEMM_ERR_TIMEOUT", 7: "SPGEMM_ERR_STATE",
    8: "SPGEMM_ERR_UNSORTED", 9: "SPGEMM_ERR_MISMATCH", 10: "SPGEMM_ERR_SCRATCH_LIMIT",
}
CLASS_NAMES = ("M1", "M2", "W", "B", "G")


class SpgemmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        self.name = SPGEMM_STATUS.get(code, str(code))
        super().__init__(f"{where}: {self.name} ({error_string(code) if _lib else code})")


class spgemm_csr_t(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class spgemm_options_t(ctypes.Structure):
    _fields_ = [("merge_max_k", ctypes.c_int32), ("m1_max_u", ctypes.c_int32), ("m2_max_u", ctypes.c_int32),
                ("warp_max_u", ctypes.c_int32), ("block_max_u", ctypes.c_int32), ("dense_slabs", ctypes.c_int32),
                ("validate", ctypes.c_int32), ("merge_values", ctypes.c_int32), ("a_storage", ctypes.c_int32),
                ("b_storage", ctypes.c_int32), ("warp_bitvec_ratio", ctypes.c_int32), ("warp_order", ctypes.c_int32),
                ("debug_spin_limit", ctypes.c_int32), ("debug_drop_tile", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class spgemm_info_t(ctypes.Structure):
    _fields_ = [("products", ctypes.c_int64), ("nnz_c", ctypes.c_int64), ("max_row_products", ctypes.c_int32),
                ("rows_per_class", ctypes.c_int32 * 5)]


def library_path() -> str:
    return _build.LIB


def load():
    """Load the CUDA library (built in-tree); raises if it is missing."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"SpGEMM CUDA library not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        lib.spgemm_workspace_size.argtypes = [P(spgemm_csr_t), P(spgemm_csr_t), P(spgemm_options_t),
                                              P(ctypes.c_size_t)]
        lib.spgemm_plan.argtypes = [P(vp), P(spgemm_csr_t), P(spgemm_csr_t), P(spgemm_options_t), vp,
                                    ctypes.c_size_t, vp]
        lib.spgemm_symbolic.argtypes = [vp, vp, P(ctypes.c_int64), vp]
        lib.spgemm_numeric.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.spgemm_compute.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int64, P(ctypes.c_int64), vp]
        lib.spgemm_status.argtypes = [vp, vp]
        lib.spgemm_plan_set_events.argtypes = [vp, vp, vp]
        lib.spgemm_compute_async.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int64, vp, vp]
        lib.spgemm_backward_workspace_size.argtypes = [P(spgemm_csr_t), P(spgemm_csr_t), P(ctypes.c_size_t)]
        lib.spgemm_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        lib.spgemm_plan_info.argtypes = [vp, P(spgemm_info_t)]
        lib.spgemm_free.argtypes = [vp]
        lib.spgemm_scan_counts_noalloc.argtypes = [vp, ctypes.c_int64, P(ctypes.c_int64), vp]
        lib.spgemm_replay_size.argtypes = [vp, P(ctypes.c_size_t)]
        lib.spgemm_replay_record.argtypes = [vp, vp, vp, ctypes.c_size_t, vp]
        lib.spgemm_replay.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.spgemm_multiply.argtypes = [P(spgemm_csr_t), P(spgemm_csr_t), P(spgemm_options_t), vp, ctypes.c_size_t,
                                        vp, vp, vp, ctypes.c_int64, P(ctypes.c_int64), P(ctypes.c_int64), vp]
        lib.spgemm_multiply_async.argtypes = [P(spgemm_csr_t), P(spgemm_csr_t), P(spgemm_options_t), vp,
                                              ctypes.c_size_t, vp, vp, vp, ctypes.c_int64, vp]
        lib.spgemm_multiply_result.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_int64), vp]
        lib.spgemm_error_string.argtypes = [ctypes.c_int]
        lib.spgemm_error_string.restype = ctypes.c_char_p
        lib.spgemm_version.restype = ctypes.c_int32
        for name in ("spgemm_workspace_size", "spgemm_plan", "spgemm_symbolic", "spgemm_numeric",
                     "spgemm_compute", "spgemm_status", "spgemm_plan_info", "spgemm_free",
                     "spgemm_plan_set_events", "spgemm_compute_async", "spgemm_backward_workspace_size",
                     "spgemm_backward", "spgemm_scan_counts_noalloc", "spgemm_replay_size",
                     "spgemm_replay_record", "spgemm_replay", "spgemm_multiply", "spgemm_multiply_async",
                     "spgemm_multiply_result"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def error_string(code: int) -> str:
    return load().spgemm_error_string(int(code)).decode()


def _check(code: int, where: str):
    if code != 0:
        raise SpgemmError(code, where)


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None or t.numel() == 0:
        return None
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


@dataclass
class DeviceCSR:
    """CSR matrix in device memory: int32 row_ptr/col_idx, float64 val (torch tensors)."""

    rows: int
    cols: int
    row_ptr: torch.Tensor
    col_idx: torch.Tensor
    val: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.col_idx.numel())

    @staticmethod
    def from_host(M, device="cuda") -> "DeviceCSR":
        return DeviceCSR(M.rows, M.cols,
                         torch.from_numpy(np.ascontiguousarray(M.row_ptr, np.int32)).to(device),
                         torch.from_numpy(np.ascontiguousarray(M.col_idx, np.int32)).to(device),
                         torch.from_numpy(np.ascontiguousarray(M.val, np.float64)).to(device))

    def desc(self, with_values: bool = True) -> spgemm_csr_t:
        return spgemm_csr_t(self.rows, self.cols, self.nnz, _ptr(self.row_ptr), _ptr(self.col_idx),
                            _ptr(self.val) if with_values else None)

    def to_host(self) -> dict:
        return dict(rows=self.rows, cols=self.cols, row_ptr=self.row_ptr.cpu().numpy(),
                    col_idx=self.col_idx.cpu().numpy(), val=self.val.cpu().numpy(), nnz=self.nnz)


@dataclass
class DeviceCSC:
    """Matrix in compressed columns in device memory: int32 col_ptr (cols + 1), int32 row_idx, float64
    val.  Passed to the library with the option a_storage / b_storage = 1 (the descriptor keeps the
    matrix's own rows and cols; its row_ptr and col_idx fields carry col_ptr and row_idx)."""

    rows: int
    cols: int
    col_ptr: torch.Tensor
    row_idx: torch.Tensor
    val: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.row_idx.numel())

    def desc(self, with_values: bool = True) -> spgemm_csr_t:
        return spgemm_csr_t(self.rows, self.cols, self.nnz, _ptr(self.col_ptr), _ptr(self.row_idx),
                            _ptr(self.val) if with_values else None)


def with_storage(A, B, opt: spgemm_options_t | None = None) -> spgemm_options_t | None:
    """opt (copied) with a_storage / b_storage set for operands given as DeviceCSC."""
    a, b = isinstance(A, DeviceCSC), isinstance(B, DeviceCSC)
    if not (a or b or (opt is not None and (opt.a_storage or opt.b_storage))):
        return opt
    o = spgemm_options_t.from_buffer_copy(opt) if opt is not None else spgemm_options_t()
    o.a_storage, o.b_storage = int(a), int(b)
    return o


def options(**kw) -> spgemm_options_t:
    o = spgemm_options_t()
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


# ---- thin wrappers with the C names --------------------------------------------------------

def spgemm_workspace_size(A: DeviceCSR, B: DeviceCSR, opt: spgemm_options_t | None = None) -> int:
    n = ctypes.c_size_t(0)
    a, b = A.desc(False), B.desc(False)
    _check(load().spgemm_workspace_size(ctypes.byref(a), ctypes.byref(b), ctypes.byref(opt) if opt else None,
                                        ctypes.byref(n)), "spgemm_workspace_size")
    return int(n.value)


def spgemm_plan(A: DeviceCSR, B: DeviceCSR, workspace: torch.Tensor, opt: spgemm_options_t | None = None,
                stream=None) -> int:
    h = ctypes.c_void_p(0)
    a, b = A.desc(False), B.desc(False)
    _check(load().spgemm_plan(ctypes.byref(h), ctypes.byref(a), ctypes.byref(b),
                              ctypes.byref(opt) if opt else None, workspace.data_ptr(),
                              workspace.numel() * workspace.element_size(), _stream(stream)), "spgemm_plan")
    return h.value


def spgemm_symbolic(plan: int, C_row_ptr: torch.Tensor, stream=None) -> int:
    nnz = ctypes.c_int64(0)
    _check(load().spgemm_symbolic(plan, C_row_ptr.data_ptr(), ctypes.byref(nnz), _stream(stream)),
           "spgemm_symbolic")
    return int(nnz.value)


def spgemm_numeric(plan: int, A_val: torch.Tensor, B_val: torch.Tensor, C_col: torch.Tensor, C_val: torch.Tensor,
                   stream=None):
    _check(load().spgemm_numeric(plan, _ptr(A_val), _ptr(B_val), _ptr(C_col), _ptr(C_val), _stream(stream)),
           "spgemm_numeric")


def spgemm_compute(plan: int, A_val: torch.Tensor, B_val: torch.Tensor, C_row_ptr: torch.Tensor,
                   C_col: torch.Tensor, C_val: torch.Tensor, stream=None) -> int:
    nnz = ctypes.c_int64(0)
    cap = min(C_col.numel(), C_val.numel())
    _check(load().spgemm_compute(plan, _ptr(A_val), _ptr(B_val), C_row_ptr.data_ptr(), _ptr(C_col), _ptr(C_val),
                                 cap, ctypes.byref(nnz), _stream(stream)), "spgemm_compute")
    return int(nnz.value)


def spgemm_compute_async(plan: int, A_val: torch.Tensor, B_val: torch.Tensor, C_row_ptr: torch.Tensor,
                         C_col: torch.Tensor, C_val: torch.Tensor, nnz_device: torch.Tensor | None = None,
                         stream=None):
    """Enqueue the single-pass product without synchronising (CUDA-graph capturable)."""
    cap = min(C_col.numel(), C_val.numel())
    _check(load().spgemm_compute_async(plan, _ptr(A_val), _ptr(B_val), C_row_ptr.data_ptr(), _ptr(C_col),
                                       _ptr(C_val), cap, _ptr(nnz_device), _stream(stream)), "spgemm_compute_async")


def spgemm_backward_workspace_size(A: DeviceCSR, B: DeviceCSR) -> int:
    n = ctypes.c_size_t(0)
    a, b = A.desc(False), B.desc(False)
    _check(load().spgemm_backward_workspace_size(ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)),
           "spgemm_backward_workspace_size")
    return int(n.value)


def spgemm_backward(plan: int, A_val, B_val, dC_val, dA_val=None, dB_val=None, workspace=None, stream=None):
    """dA = (dC B^T) on A's structure and dB = (A^T dC) on B's structure (either may be None)."""
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(load().spgemm_backward(plan, _ptr(A_val), _ptr(B_val), _ptr(dC_val), _ptr(dA_val), _ptr(dB_val),
                                  _ptr(workspace), ws_bytes, _stream(stream)), "spgemm_backward")


def spgemm_status(plan: int, stream=None):
    _check(load().spgemm_status(plan, _stream(stream)), "spgemm_status")


def spgemm_plan_info(plan: int) -> dict:
    info = spgemm_info_t()
    _check(load().spgemm_plan_info(plan, ctypes.byref(info)), "spgemm_plan_info")
    return dict(products=int(info.products), nnz_c=int(info.nnz_c), max_row_products=int(info.max_row_products),
                rows_per_class=dict(zip(CLASS_NAMES, list(info.rows_per_class))))


def spgemm_plan_set_events(plan: int, start=None, stop=None):
    """Record torch.cuda.Event objects (timing enabled) around the plan's compute kernels."""
    # torch creates the CUDA event on its first record(): record once so the handles exist
    for ev in (start, stop):
        if ev is not None and not ev.cuda_event:
            ev.record()
    _check(load().spgemm_plan_set_events(plan, start.cuda_event if start is not None else None,
                                         stop.cuda_event if stop is not None else None), "spgemm_plan_set_events")


def spgemm_free(plan: int):
    if plan:
        load().spgemm_free(plan)


def spgemm_replay_size(plan: int) -> int:
    n = ctypes.c_size_t(0)
    _check(load().spgemm_replay_size(plan, ctypes.byref(n)), "spgemm_replay_size")
    return int(n.value)


def spgemm_replay_record(plan: int, C_col: torch.Tensor, map_buf: torch.Tensor, stream=None):
    _check(load().spgemm_replay_record(plan, _ptr(C_col), map_buf.data_ptr(), map_buf.numel() * map_buf.element_size(),
                                       _stream(stream)), "spgemm_replay_record")


def spgemm_replay(plan: int, A_val: torch.Tensor, B_val: torch.Tensor, map_buf: torch.Tensor, C_col: torch.Tensor,
                  C_val: torch.Tensor, stream=None):
    _check(load().spgemm_replay(plan, _ptr(A_val), _ptr(B_val), map_buf.data_ptr(), _ptr(C_col), _ptr(C_val),
                                _stream(stream)), "spgemm_replay")


def spgemm_multiply(A, B, C_row_ptr: torch.Tensor, C_col: torch.Tensor, C_val: torch.Tensor, workspace: torch.Tensor,
                    opt: spgemm_options_t | None = None, stream=None, raise_on_overflow: bool = True):
    """Plan + single-pass product in one call (one host synchronisation); C's capacity is
    min(C_col.numel(), C_val.numel()).  Returns (nnz(C), F).  With raise_on_overflow=False an
    OVERFLOW (capacity below nnz(C)) returns (nnz(C), F) too, so the caller can resize C to F."""
    opt = with_storage(A, B, opt)
    a, b = A.desc(True), B.desc(True)
    nnz, F = ctypes.c_int64(0), ctypes.c_int64(0)
    cap = min(C_col.numel(), C_val.numel())
    code = load().spgemm_multiply(ctypes.byref(a), ctypes.byref(b), ctypes.byref(opt) if opt else None,
                                  workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                  C_row_ptr.data_ptr(), _ptr(C_col), _ptr(C_val), cap, ctypes.byref(nnz),
                                  ctypes.byref(F), _stream(stream))
    if code == 3 and not raise_on_overflow:
        return int(nnz.value), int(F.value)
    _check(code, "spgemm_multiply")
    return int(nnz.value), int(F.value)


def spgemm_multiply_async(A, B, C_row_ptr: torch.Tensor, C_col: torch.Tensor, C_val: torch.Tensor,
                          workspace: torch.Tensor, opt: spgemm_options_t | None = None, stream=None):
    """Enqueue spgemm_multiply's work without synchronising (CUDA-graph capturable); read the result
    with spgemm_multiply_result(workspace)."""
    opt = with_storage(A, B, opt)
    a, b = A.desc(True), B.desc(True)
    cap = min(C_col.numel(), C_val.numel())
    _check(load().spgemm_multiply_async(ctypes.byref(a), ctypes.byref(b), ctypes.byref(opt) if opt else None,
                                        workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                        C_row_ptr.data_ptr(), _ptr(C_col), _ptr(C_val), cap, _stream(stream)),
           "spgemm_multiply_async")


def spgemm_multiply_result(workspace: torch.Tensor, stream=None, raise_on_overflow: bool = True):
    """(nnz(C), F) left in the workspace by the last spgemm_multiply_async on it (synchronises)."""
    nnz, F = ctypes.c_int64(0), ctypes.c_int64(0)
    code = load().spgemm_multiply_result(workspace.data_ptr(), ctypes.byref(nnz), ctypes.byref(F), _stream(stream))
    if not (code == 3 and not raise_on_overflow):
        _check(code, "spgemm_multiply_result")
    return int(nnz.value), int(F.value)


class GraphProduct:
    """C = A*B for arrays whose shapes stay fixed, from a CUDA graph of spgemm_multiply_async: each
    run() replays binning and the single-pass product over the arrays' current contents (no host
    work between its kernels) and reads nnz(C) and F back once.  C holds `capacity` entries."""

    def __init__(self, A, B, capacity: int, opt: spgemm_options_t | None = None):
        self.A, self.B, self.opt = A, B, with_storage(A, B, opt)
        dev = A.val.device
        self.ws = torch.empty(spgemm_workspace_size(A, B, self.opt), dtype=torch.uint8, device=dev)
        self.C_row_ptr = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
        self.C_col = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
        self.C_val = torch.empty(max(capacity, 1), dtype=torch.float64, device=dev)
        self._enqueue()                       # eager: kernel attributes set before the capture
        spgemm_multiply_result(self.ws, raise_on_overflow=False)
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=side):
            self._enqueue()
        torch.cuda.current_stream(dev).wait_stream(side)

    def _enqueue(self):
        spgemm_multiply_async(self.A, self.B, self.C_row_ptr, self.C_col, self.C_val, self.ws, self.opt)

    def run(self, raise_on_overflow: bool = True):
        """Replay; returns (nnz(C), F)."""
        self.graph.replay()
        return spgemm_multiply_result(self.ws, raise_on_overflow=raise_on_overflow)


def multiply_once(A, B, opt: spgemm_options_t | None = None, stream=None, capacity: int | None = None,
                  workspace: torch.Tensor | None = None) -> DeviceCSR:
    """C = A*B through spgemm_multiply: one call, one host synchronisation when `capacity` (default
    nnz(A) + nnz(B) + rows of A) holds C; otherwise a second call with C sized by F."""
    opt = with_storage(A, B, opt)
    dev = A.val.device
    need = spgemm_workspace_size(A, B, opt)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    cap = max(capacity if capacity is not None else A.nnz + B.nnz + A.rows, 1)
    C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
    C_col = torch.empty(cap, dtype=torch.int32, device=dev)
    C_val = torch.empty(cap, dtype=torch.float64, device=dev)
    nnz, F = spgemm_multiply(A, B, C_rp, C_col, C_val, workspace, opt, stream, raise_on_overflow=False)
    if nnz > cap:
        C_col = torch.empty(max(F, 1), dtype=torch.int32, device=dev)
        C_val = torch.empty(max(F, 1), dtype=torch.float64, device=dev)
        nnz, F = spgemm_multiply(A, B, C_rp, C_col, C_val, workspace, opt, stream)
    return DeviceCSR(A.rows, B.cols, C_rp, C_col[:nnz], C_val[:nnz])


def spgemm_scan_counts_noalloc(row_ptr: torch.Tensor, rows: int | None = None, stream=None) -> int:
    """In place: per-row counts in row_ptr[:rows] -> row pointers in row_ptr[:rows + 1]; returns the
    total.  Uses the library's fixed scratch array, so nothing is allocated; calls must not overlap."""
    if rows is None:
        rows = row_ptr.numel() - 1
    if row_ptr.dtype != torch.int32 or not row_ptr.is_cuda or not row_ptr.is_contiguous():
        raise ValueError("row_ptr must be a contiguous int32 CUDA tensor")
    if rows + 1 > row_ptr.numel():
        raise ValueError(f"row_ptr holds {row_ptr.numel()} entries, fewer than rows + 1 = {rows + 1}")
    total = ctypes.c_int64(0)
    _check(load().spgemm_scan_counts_noalloc(row_ptr.data_ptr() if row_ptr.numel() else None, int(rows),
                                             ctypes.byref(total), _stream(stream)), "spgemm_scan_counts_noalloc")
    return total.value


# ---- the whole product ----------------------------------------------------------------------

class Product:
    """One planned product C = A*B: workspace, plan, C's row pointer; numeric is repeatable."""

    def __init__(self, A: DeviceCSR, B: DeviceCSR, opt: spgemm_options_t | None = None, stream=None,
                 workspace: torch.Tensor | None = None):
        if A.cols != B.rows:
            raise ValueError("inner dimensions differ")
        opt = with_storage(A, B, opt)
        self.A, self.B, self.opt = A, B, opt
        dev = A.val.device
        need = spgemm_workspace_size(A, B, opt)
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(need, dtype=torch.uint8, device=dev)
        self.workspace = workspace
        self.plan = spgemm_plan(A, B, workspace, opt, stream)
        self.C_row_ptr = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
        self.nnz = spgemm_symbolic(self.plan, self.C_row_ptr, stream)
        self.info = spgemm_plan_info(self.plan)

    def numeric(self, A_val=None, B_val=None, C_col=None, C_val=None, stream=None) -> DeviceCSR:
        dev = self.A.val.device
        A_val = self.A.val if A_val is None else A_val
        B_val = self.B.val if B_val is None else B_val
        if C_col is None:
            C_col = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        if C_val is None:
            C_val = torch.empty(self.nnz, dtype=torch.float64, device=dev)
        spgemm_numeric(self.plan, A_val, B_val, C_col, C_val, stream)
        return DeviceCSR(self.A.rows, self.B.cols, self.C_row_ptr, C_col, C_val)

    def record(self, C: DeviceCSR, stream=None):
        """Record the position map of C's structure (a result of numeric) for replay()."""
        self.map = torch.empty(spgemm_replay_size(self.plan), dtype=torch.uint8, device=self.A.val.device)
        spgemm_replay_record(self.plan, C.col_idx, self.map, stream)
        self.C_col = C.col_idx

    def replay(self, A_val, B_val, C_val=None, stream=None) -> DeviceCSR:
        """C's values for new values of A and B, through the recorded map (same bits as numeric)."""
        if C_val is None:
            C_val = torch.empty(self.nnz, dtype=torch.float64, device=self.A.val.device)
        spgemm_replay(self.plan, A_val, B_val, self.map, self.C_col, C_val, stream)
        return DeviceCSR(self.A.rows, self.B.cols, self.C_row_ptr, self.C_col, C_val)

    def close(self):
        if getattr(self, "plan", None):
            spgemm_free(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def multiply(A: DeviceCSR, B: DeviceCSR, opt: spgemm_options_t | None = None, stream=None,
             check: bool = False) -> DeviceCSR:
    """C = A*B on the GPU through plan / symbolic / numeric."""
    prod = Product(A, B, opt, stream)
    try:
        C = prod.numeric(stream=stream)
        if check:
            spgemm_status(prod.plan, stream)
        return C
    finally:
        prod.close()


def multiply_fused(A: DeviceCSR, B: DeviceCSR, opt: spgemm_options_t | None = None, stream=None,
                   workspace: torch.Tensor | None = None, trim: bool = True) -> DeviceCSR:
    """C = A*B through plan and the single-pass spgemm_compute (C sized by the multiplication count)."""
    opt = with_storage(A, B, opt)
    dev = A.val.device
    need = spgemm_workspace_size(A, B, opt)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    plan = spgemm_plan(A, B, workspace, opt, stream)
    try:
        F = spgemm_plan_info(plan)["products"]
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
        C_col = torch.empty(max(F, 1), dtype=torch.int32, device=dev)
        C_val = torch.empty(max(F, 1), dtype=torch.float64, device=dev)
        nnz = spgemm_compute(plan, A.val, B.val, C_rp, C_col, C_val, stream)
    finally:
        spgemm_free(plan)
    if trim:
        C_col, C_val = C_col[:nnz], C_val[:nnz]
    return DeviceCSR(A.rows, B.cols, C_rp, C_col, C_val)


# ---- torch front door ------------------------------------------------------------------------

def _from_torch(M: torch.Tensor, name: str):
    """A torch sparse CSR or CSC tensor (CUDA, int32 indices, float64 values) as a DeviceCSR/DeviceCSC."""
    if not isinstance(M, torch.Tensor) or M.layout not in (torch.sparse_csr, torch.sparse_csc):
        raise TypeError(f"{name} must be a torch.sparse_csr_tensor or torch.sparse_csc_tensor")
    if M.dim() != 2:
        raise ValueError(f"{name} must be a 2-D matrix (batched sparse tensors are not supported)")
    if not M.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    rows, cols = M.shape
    if M.layout == torch.sparse_csr:
        ptr, idx = M.crow_indices(), M.col_indices()
    else:
        ptr, idx = M.ccol_indices(), M.row_indices()
    val = M.values()
    if ptr.dtype != torch.int32 or idx.dtype != torch.int32:
        raise TypeError(f"{name} must have int32 indices (build it with crow/col index tensors of dtype int32)")
    if val.dtype != torch.float64:
        raise TypeError(f"{name} must have float64 values")
    ptr, idx, val = ptr.contiguous(), idx.contiguous(), val.contiguous()
    if M.layout == torch.sparse_csr:
        return DeviceCSR(rows, cols, ptr, idx, val)
    return DeviceCSC(rows, cols, ptr, idx, val)


def spgemm(A: torch.Tensor, B: torch.Tensor, opt: spgemm_options_t | None = None, stream=None) -> torch.Tensor:
    """C = A @ B for sparse matrices on a CUDA device; returns a torch.sparse_csr_tensor.

    A and B are torch.sparse_csr_tensor or torch.sparse_csc_tensor (any mix), int32 indices, float64
    values, any shapes with A.shape[1] == B.shape[0].  An operand in CSC is converted to rows inside
    the library (Section IV-A's storage-order conversion).  C's rows are sorted by column, with every
    structural entry kept, and C is computed by spgemm_plan + spgemm_compute (C sized by the
    multiplication count, then trimmed).  For gradients with respect to the values, use
    autograd.SpGEMMFunction."""
    a, b = _from_torch(A, "A"), _from_torch(B, "B")
    if a.cols != b.rows:
        raise ValueError(f"inner dimensions differ: A is {a.rows}x{a.cols}, B is {b.rows}x{b.cols}")
    C = multiply_fused(a, b, opt, stream)
    return torch.sparse_csr_tensor(C.row_ptr, C.col_idx, C.val, size=(a.rows, b.cols))
