"""Batches of independent products C_p = A_p * B_p in one pass.

A batch is the block-diagonal product diag(A_1..A_P) * diag(B_1..B_P) = diag(C_1..C_P): rows of
A_p only reach rows of B_p, so one plan and one single-pass launch serve every problem, with the
warps of that launch taking tiles of any problem as they free up.  After planning (which reads
back the multiplication count to size C), the whole pipeline is enqueued without host
synchronisation and captured in a CUDA graph; replaying the graph recomputes the batch.

concat(problems)          -- host: stack the problems into block-diagonal CSR matrices.
BatchedProduct(A, B)      -- device: plan, C buffers, CUDA graph of spgemm_compute_async.
per_matrix(problems)      -- device: the same products one at a time (plan + compute each), for
                             comparison.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import binding
from .synth import CSR


@dataclass
class BatchLayout:
    a_row: np.ndarray    # problem p owns rows a_row[p]:a_row[p+1] of A (and of C)
    b_row: np.ndarray    # ... rows b_row[p]:b_row[p+1] of B (= columns of A's block)
    c_col: np.ndarray    # ... columns c_col[p]:c_col[p+1] of B and C


def concat(problems) -> tuple[CSR, CSR, BatchLayout]:
    """Block-diagonal A and B of a list of (A_p, B_p) host CSR pairs."""
    P = len(problems)
    a_row = np.zeros(P + 1, np.int64)
    b_row = np.zeros(P + 1, np.int64)
    c_col = np.zeros(P + 1, np.int64)
    for t, (A, B) in enumerate(problems):
        if A.cols != B.rows:
            raise ValueError(f"problem {t}: inner dimensions differ")
        a_row[t + 1] = a_row[t] + A.rows
        b_row[t + 1] = b_row[t] + B.rows
        c_col[t + 1] = c_col[t] + B.cols
    if max(a_row[-1], b_row[-1], c_col[-1]) > np.iinfo(np.int32).max:
        raise OverflowError("batch too large for int32 indices")

    def stack(mats, row_off, col_off, nrows, ncols):
        rp = [np.zeros(1, np.int64)]
        cols, vals = [], []
        base = 0
        for t, M in enumerate(mats):
            rp.append(M.row_ptr[1:].astype(np.int64) + base)
            base += int(M.row_ptr[-1]) if M.rows else 0
            cols.append(M.col_idx.astype(np.int64) + col_off[t])
            vals.append(M.val)
        rp = np.concatenate(rp)
        if rp[-1] > np.iinfo(np.int32).max:
            raise OverflowError("batch nnz exceeds int32")
        return CSR(int(nrows), int(ncols), rp.astype(np.int32),
                   np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32),
                   np.concatenate(vals) if vals else np.zeros(0))

    A_cat = stack([A for A, _ in problems], a_row, b_row, a_row[-1], b_row[-1])
    B_cat = stack([B for _, B in problems], b_row, c_col, b_row[-1], c_col[-1])
    return A_cat, B_cat, BatchLayout(a_row, b_row, c_col)


def split(C: dict, layout: BatchLayout, p: int) -> dict:
    """Problem p's block of a host result dict (row_ptr, col_idx, val): local row pointer and columns."""
    r0, r1 = int(layout.a_row[p]), int(layout.a_row[p + 1])
    rp = np.asarray(C["row_ptr"], np.int64)
    e0, e1 = int(rp[r0]), int(rp[r1])
    return dict(rows=r1 - r0, cols=int(layout.c_col[p + 1] - layout.c_col[p]), row_ptr=rp[r0:r1 + 1] - e0,
                col_idx=np.asarray(C["col_idx"][e0:e1], np.int64) - int(layout.c_col[p]),
                val=np.asarray(C["val"][e0:e1]), nnz=e1 - e0)


class BatchedProduct:
    """The batch as one plan and a CUDA graph of the single-pass product.

    run() replays the graph (values of A and B may change in place between replays; structures
    and buffers must not).  C's row pointer, columns (global, block-diagonal) and values are the
    attributes C_row_ptr, C_col, C_val; nnz() reads back nnz(C).
    """

    def __init__(self, A: binding.DeviceCSR, B: binding.DeviceCSR, opt=None, capture: bool = True):
        self.A, self.B, self.opt = A, B, opt
        dev = A.row_ptr.device
        self.ws = torch.empty(binding.spgemm_workspace_size(A, B, opt), dtype=torch.uint8, device=dev)
        self.plan = binding.spgemm_plan(A, B, self.ws, opt)
        self.info = binding.spgemm_plan_info(self.plan)
        F = max(self.info["products"], 1)
        self.C_row_ptr = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
        self.C_col = torch.empty(F, dtype=torch.int32, device=dev)
        self.C_val = torch.empty(F, dtype=torch.float64, device=dev)
        self.nnz_dev = torch.zeros(1, dtype=torch.int64, device=dev)
        self.graph = None
        # one eager run (sets kernel attributes, checks the status), then capture
        self._enqueue()
        binding.spgemm_status(self.plan)
        if capture:
            side = torch.cuda.Stream(device=dev)
            side.wait_stream(torch.cuda.current_stream(dev))
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=side):
                self._enqueue()
            torch.cuda.current_stream(dev).wait_stream(side)

    def _enqueue(self):
        binding.spgemm_compute_async(self.plan, self.A.val, self.B.val, self.C_row_ptr, self.C_col, self.C_val,
                                     self.nnz_dev)

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._enqueue()

    def nnz(self) -> int:
        return int(self.nnz_dev.item())

    def check(self):
        binding.spgemm_status(self.plan)

    def result_host(self) -> dict:
        n = self.nnz()
        return dict(rows=self.A.rows, cols=self.B.cols, row_ptr=self.C_row_ptr.cpu().numpy(),
                    col_idx=self.C_col[:n].cpu().numpy(), val=self.C_val[:n].cpu().numpy(), nnz=n)

    def close(self):
        if getattr(self, "plan", None):
            self.graph = None
            binding.spgemm_free(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PerMatrix:
    """The same products one at a time: each problem planned and computed on its own (host
    synchronisation for the multiplication count and for nnz(C) in every call)."""

    def __init__(self, problems_dev, opt=None):
        self.items = []
        for A, B in problems_dev:
            ws = torch.empty(binding.spgemm_workspace_size(A, B, opt), dtype=torch.uint8, device=A.row_ptr.device)
            C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device=A.row_ptr.device)
            self.items.append((A, B, ws, C_rp))
        self.opt = opt
        self.F = None

    def run(self):
        F = 0
        for A, B, ws, C_rp in self.items:
            plan = binding.spgemm_plan(A, B, ws, self.opt)
            try:
                f = binding.spgemm_plan_info(plan)["products"]
                F += f
                C_col = torch.empty(max(f, 1), dtype=torch.int32, device=A.row_ptr.device)
                C_val = torch.empty(max(f, 1), dtype=torch.float64, device=A.row_ptr.device)
                binding.spgemm_compute(plan, A.val, B.val, C_rp, C_col, C_val)
            finally:
                binding.spgemm_free(plan)
        self.F = F


def main(argv=None):
    """Replay the batch of `synth.batch_problems` as one block-diagonal product and report the
    time per replay (CUDA events).  python -m paper_1303_1651_gb300.batched [--count 512] [--replays 5]"""
    import argparse
    import json
    from . import synth
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--seed", type=int, default=synth.SEED_BATCH)
    ap.add_argument("--replays", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    args = ap.parse_args(argv)
    A, B, _ = concat(synth.batch_problems(count=args.count, seed=args.seed))
    dev = torch.device("cuda", 0)
    dA, dB = binding.DeviceCSR.from_host(A, dev), binding.DeviceCSR.from_host(B, dev)
    bp = BatchedProduct(dA, dB)
    for _ in range(args.warmup):
        bp.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.replays):
        bp.run()
    e1.record()
    torch.cuda.synchronize()
    bp.check()
    ms = e0.elapsed_time(e1) / max(args.replays, 1)
    print(json.dumps({"problems": args.count, "rows": A.rows, "products": bp.info["products"],
                      "rows_per_class": bp.info["rows_per_class"], "ms_per_replay": ms,
                      "gflops": 2 * bp.info["products"] / (ms * 1e-3) / 1e9}))
    bp.close()


if __name__ == "__main__":
    main()
