#!/usr/bin/env python
"""SpGEMM benchmark: C = A*B on CSR (int32 indices, float64 values), GFLOP/s and % of HBM roofline.

Workload (one step = the whole pipeline -- binning, symbolic, scan, numeric --
for both products, inputs resident in HBM, C buffers from torch's caching
allocator, nnz(C) read back to the host as the C ABI requires):
  * laplacian5_2048_sq : A = 5-point Laplacian on a 2048 x 2048 grid (4.19M rows), C = A*A
  * random_1M_k8       : A, B 1M x 1M, 8 distinct uniform columns per row, U(-1,1), C = A*B
Flops are 2 per multiplication (Section III of the paper).  Inputs total
~2.5 GB per step, larger than L2, so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain Gustavson of oracle/) on the
host, on a row sample of the same workload, and prints the same JSON line.
Under torchrun (N > 1) every rank runs its own replica of the workload (weak
scaling, no collective on the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1303_1651_gb300 import roofline, synth  # noqa: E402

METRIC = "SpGEMM GFLOP/s (2/intermediate product) and % HBM roofline; batched vs plain"
WORKLOAD = "plain_large: laplacian5_2048_sq + random_1M_k8"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain", choices=["plain", "medium", "small", "batched16"],
                    help="plain: the benchmark workload; small: Laplacian 64^2 + random 4096 x 8 (the small "
                         "case); medium: Laplacian 1024^2 + random 500K x 8 "
                         "(inputs above L2, a few hundred MB; for profiler captures); batched16: the first "
                         "16 random x random problems of the batched workload as one block-diagonal product "
                         "(for captures of the warp-per-row class)")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched, backward and long-row measurements")
    ap.add_argument("--no-parity", action="store_true", help="skip the full-size check against the oracle")
    ap.add_argument("--sweep", action="store_true",
                    help="time the size sweep instead (13 log-spaced N from 1e3 to 1e7 for the Laplacian^2 and "
                         "random*random at 4, 8 and 16 per row; one JSON line with a row per point)")
    ap.add_argument("--verbose", action="store_true")
    return ap.parse_args()


def make_workload(kind: str = "plain"):
    if kind == "batched16":
        from paper_1303_1651_gb300 import batched
        probs = synth.batch_problems(count=512, seed=synth.SEED_BATCH)[256:272]
        A, B, _ = batched.concat(probs)
        return [("batched16_random", A, B)]
    if kind == "small":
        L = synth.laplacian5(64)
        return [("laplacian5_64_sq", L, L), ("random_4096_k8", synth.random_k(4096, 8, synth.SEED_A),
                                             synth.random_k(4096, 8, synth.SEED_B))]
    if kind == "medium":
        L = synth.laplacian5(1024)
        R1 = synth.random_k(500_000, 8, synth.SEED_A)
        R2 = synth.random_k(500_000, 8, synth.SEED_B)
        return [("laplacian5_1024_sq", L, L), ("random_500K_k8", R1, R2)]
    L = synth.laplacian5(2048)
    R1 = synth.random_k(1_000_000, 8, synth.SEED_A)
    R2 = synth.random_k(1_000_000, 8, synth.SEED_B)
    return [("laplacian5_2048_sq", L, L), ("random_1M_k8", R1, R2)]


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def hbm_peak():
    p = peaks()
    if p and p.get("hbm_gbs"):
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """Hash of the fused kernels' code (comments and blank lines left out, so that only a change of
    the code itself invalidates the stored DRAM traffic)."""
    h = hashlib.sha256()
    for f in ("common.cuh", "merge.cu"):
        for line in open(os.path.join(ROOT, "paper_1303_1651_gb300", "csrc", f)).read().splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def committed_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernel source."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        e = t.get(kernel)
        if e and e.get("source_hash") == kernel_source_hash():
            return int(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.lines, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def sm_median(self, start: int = 0):
        """Median SM clock of the samples from index start on (None if there are none)."""
        v = []
        for ln in self.lines[start:]:
            try:
                v.append(float(ln.split(",")[0]))
            except ValueError:
                continue
        return float(np.median(v)) if v else None

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0])); mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------------------------
# reference arm: the CPU oracle on a row sample of the workload
# ----------------------------------------------------------------------------------------------

def row_sample(A, frac: float):
    m = max(1, int(A.rows * frac))
    nnz = int(A.row_ptr[m])
    return synth.CSR(m, A.cols, A.row_ptr[:m + 1].copy(), A.col_idx[:nnz].copy(), A.val[:nnz].copy())


def oracle_rate(work, frac: float, reps: int = 1):
    import oracle
    F = 0
    t0 = time.perf_counter()
    for _ in range(reps):
        for _, A, B in work:
            As = row_sample(A, frac)
            F += oracle.spgemm(As, B)["F"]
    dt = time.perf_counter() - t0
    return 2 * F / dt / 1e9, dt, F


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model")):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_protocol(work, frac: float, min_s: float = 2.0, min_runs: int = 5, max_s: float = 15.0) -> dict:
    """The oracle on one host thread, on the first frac of the rows of each product, repeated until
    at least min_s seconds and min_runs runs (the paper's protocol, Section III): best and median."""
    rates, total = [], 0.0
    F = 0
    while (total < min_s or len(rates) < min_runs) and total < max_s:
        r, dt, F = oracle_rate(work, frac)
        rates.append(r)
        total += dt
    return {"value": max(rates), "median": float(np.median(rates)), "unit": "GFLOP/s", "cores": 1, "threads": 1,
            "kind": "oracle", "runs": len(rates), "seconds": round(total, 2), "cpu_model": cpu_model(),
            "sample": f"first {frac:.4g} of the rows of A in each product, full B ({F} products per run); "
                      f"best of {len(rates)} runs"}


# Worker side of the multi-process oracle: each worker builds the (seeded) workload once.
_WORK = {}


def _worker_work(kind):
    if kind not in _WORK:
        _WORK.clear()
        _WORK[kind] = make_workload(kind)
    return _WORK[kind]


def _oracle_rows(kind, i, r0, r1):
    """Oracle product of rows r0..r1 of product i of the workload: (products, seconds)."""
    import oracle
    _, A, B = _worker_work(kind)[i]
    As = row_block(A, r0, r1)
    t0 = time.perf_counter()
    F = oracle.spgemm(As, B)["F"]
    return F, time.perf_counter() - t0


def _oracle_check_rows(kind, name, r0, r1, rp, col, val):
    """Rows r0..r1 of the named product computed on the GPU (rp relative to its first entry) against
    the oracle: (pattern equal, max |c - c_ref| / sum|a b|, max plain relative error over c_ref != 0)."""
    import oracle
    _, A, B = next(w for w in _worker_work(kind) if w[0] == name)
    R = oracle.spgemm(row_block(A, r0, r1), B)
    same = np.array_equal(np.asarray(rp, np.int64), R["row_ptr"]) and np.array_equal(np.asarray(col, np.int64),
                                                                                     R["col_idx"])
    if not same:
        return False, float("inf"), float("inf")
    diff = np.abs(np.asarray(val) - R["val"])
    gate = float((diff / np.where(R["absval"] > 0, R["absval"], 1.0)).max(initial=0.0))
    nz = R["val"] != 0
    plain = float((diff[nz] / np.abs(R["val"][nz])).max(initial=0.0))
    return True, gate, plain


def row_block(A, r0: int, r1: int):
    """Rows r0..r1-1 of A (all its columns)."""
    e0, e1 = int(A.row_ptr[r0]), int(A.row_ptr[r1])
    return synth.CSR(r1 - r0, A.cols, (A.row_ptr[r0:r1 + 1] - e0).astype(np.int32), A.col_idx[e0:e1].copy(),
                     A.val[e0:e1].copy())


def chunks(rows: int, n: int):
    step = max(1, -(-rows // n))
    return [(r, min(rows, r + step)) for r in range(0, rows, step)]


def spawn_pool(workers: int):
    """A process pool started with spawn (safe after CUDA has been initialised in this process)."""
    import multiprocessing
    from concurrent.futures import ProcessPoolExecutor
    return ProcessPoolExecutor(workers, mp_context=multiprocessing.get_context("spawn"))


def oracle_all_cores(kind, work, workers: int, min_s: float = 2.0, min_runs: int = 5, max_s: float = 20.0) -> dict:
    """The oracle over the whole workload on every host core: rows split into chunks, one process
    per core; best and median wall time of repeated runs."""
    jobs = [(kind, i, r0, r1) for i, (_, A, _) in enumerate(work) for r0, r1 in chunks(A.rows, 4 * workers)]
    rates, total, F = [], 0.0, 0
    with spawn_pool(workers) as ex:
        list(ex.map(_worker_work, [kind] * (4 * workers)))      # every worker builds the workload once
        while (total < min_s or len(rates) < min_runs) and total < max_s:
            t0 = time.perf_counter()
            F = sum(f for f, _ in ex.map(_oracle_rows, *zip(*jobs)))
            dt = time.perf_counter() - t0
            rates.append(2 * F / dt / 1e9)
            total += dt
    return {"value": max(rates), "median": float(np.median(rates)), "unit": "GFLOP/s", "cores": workers,
            "threads": workers, "kind": "oracle, one process per host core over row chunks", "runs": len(rates),
            "cpu_model": cpu_model(), "sample": f"the whole workload ({F} products per run); best of {len(rates)} runs"}


def check_full_products(kind, results, workers: int) -> dict:
    """Every entry of the full-size products against the oracle (rows in chunks over the host cores):
    pattern bit-exact, the gate max |c - c_ref| / sum|a b|, and the plain max relative error."""
    out = {}
    with spawn_pool(workers) as ex:
        for name, rp, col, val in results:
            jobs = []
            for r0, r1 in chunks(len(rp) - 1, 4 * workers):
                e0, e1 = int(rp[r0]), int(rp[r1])
                jobs.append(ex.submit(_oracle_check_rows, kind, name, r0, r1, rp[r0:r1 + 1] - e0, col[e0:e1],
                                      val[e0:e1]))
            res = [j.result() for j in jobs]
            out[name] = {"pattern_equal": all(r[0] for r in res),
                         "max_err_over_sum_abs": max(r[1] for r in res),
                         "max_plain_rel_err": max(r[2] for r in res), "entries": int(rp[-1])}
    return out


def combined_rate(work, threads: int, frac: float = 1.0):
    """The paper's Combined CPU kernel (Section IV-B) over the workload, or over the first frac of
    the rows of A in each product."""
    import baseline
    F = 0
    t0 = time.perf_counter()
    for _, A, B in work:
        As = A if frac >= 1.0 else row_sample(A, frac)
        F += baseline.combined(As, B, threads)["F"]
    dt = time.perf_counter() - t0
    return 2 * F / dt / 1e9, dt, F


def combined_baseline(work) -> dict:
    """The paper's own optimised CPU kernel on every host thread (whole workload) and on one (a row
    sample).  A failure to build or run it is reported in the line instead of ending the run."""
    try:
        import baseline
        threads = baseline.max_threads()
        combined_rate(work, threads, 1.0 / 64)
        rate_all, dt_all, _ = combined_rate(work, threads)
        rate_one, dt_one, _ = combined_rate(work, 1, 0.25)
    except Exception as e:  # noqa: BLE001 -- a baseline must not cost the GPU measurement
        return {"unavailable": f"{type(e).__name__}: {e}"}
    return {"value": rate_all, "unit": "GFLOP/s", "cores": threads,
            "kind": "the paper's Combined kernel (Section IV-B), C++ -O3, OpenMP over row chunks",
            "sample": f"the whole workload, one step ({dt_all:.2f} s)",
            "single_thread": {"value": rate_one, "cores": 1,
                              "sample": f"first 1/4 of the rows of A in each product, full B ({dt_one:.2f} s)"}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    work = make_workload(args.workload)
    frac = 0.25
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle_rate(work, frac / 8)
    t0 = time.perf_counter()
    F = 0
    for _ in range(args.steps):
        _, _, f = oracle_rate(work, frac)
        F += f
    dt = time.perf_counter() - t0
    value = 2 * F / dt / 1e9
    sample = f"first {int(frac * 100)}% of the rows of A in each product, full B, per step"
    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": sample, "indices": "int32 (oracle uses int64)"},
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------------

def run_numeric_only(args, prods, dev, stream, binding, torch):
    """Numeric-only timed region: plan + symbolic + record once, then K numeric passes and K replays."""
    out = {"numeric": {"ms_per_step": 0.0}, "replay": {"ms_per_step": 0.0}}
    F_total = 0
    for p in prods:
        plan = binding.spgemm_plan(p["dA"], p["dB"], p["ws"], None, stream)
        try:
            nnz = binding.spgemm_symbolic(plan, p["C_rp"], stream)
            F_total += binding.spgemm_plan_info(plan)["products"]
            C_col = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
            C_val = torch.empty(max(nnz, 1), dtype=torch.float64, device=dev)
            binding.spgemm_numeric(plan, p["dA"].val, p["dB"].val, C_col, C_val, stream)
            mp = torch.empty(binding.spgemm_replay_size(plan), dtype=torch.uint8, device=dev)
            binding.spgemm_replay_record(plan, C_col, mp, stream)
            for name, fn in (("numeric", lambda: binding.spgemm_numeric(plan, p["dA"].val, p["dB"].val, C_col, C_val,
                                                                        stream)),
                             ("replay", lambda: binding.spgemm_replay(plan, p["dA"].val, p["dB"].val, mp, C_col, C_val,
                                                                      stream))):
                for _ in range(max(args.warmup, 3)):
                    fn()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    fn()
                e1.record(stream)
                torch.cuda.synchronize()
                out[name]["ms_per_step"] += e0.elapsed_time(e1) / args.steps
            binding.spgemm_status(plan, stream)
        finally:
            binding.spgemm_free(plan)
    for name in out:
        out[name]["value"] = 2 * F_total / (out[name]["ms_per_step"] * 1e-3) / 1e9
        out[name]["unit"] = "GFLOP/s"
    out["note"] = "both products, values recomputed on a planned structure; replay uses a recorded position map"
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1303_1651_gb300 import binding, build, ranks
    build.build()
    binding.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    work = make_workload(args.workload)
    stream = torch.cuda.current_stream()
    prods = []
    for name, A, B in work:
        dA = binding.DeviceCSR.from_host(A, dev)
        dB = dA if B is A else binding.DeviceCSR.from_host(B, dev)
        ws = torch.empty(binding.spgemm_workspace_size(dA, dB), dtype=torch.uint8, device=dev)
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
        prods.append(dict(name=name, A=A, B=B, dA=dA, dB=dB, ws=ws, C_rp=C_rp,
                          ev0=[], ev1=[]))

    def one_product(p, record: bool):
        """plan (binning, F read back) -> C sized by F -> single-pass compute (nnz(C) read back)."""
        plan = binding.spgemm_plan(p["dA"], p["dB"], p["ws"], None, stream)
        try:
            info = binding.spgemm_plan_info(plan)
            F = info["products"]
            C_col = torch.empty(max(F, 1), dtype=torch.int32, device=dev)
            C_val = torch.empty(max(F, 1), dtype=torch.float64, device=dev)
            if record:
                e0, e1 = p["ev_free"].pop()
                binding.spgemm_plan_set_events(plan, e0, e1)
                p["ev0"].append(e0); p["ev1"].append(e1)
            nnz = binding.spgemm_compute(plan, p["dA"].val, p["dB"].val, p["C_rp"], C_col, C_val, stream)
            p["info"] = info
            p["nnz"] = nnz
            p["last_C"] = (C_col, C_val)
        finally:
            binding.spgemm_free(plan)
        return C_col, C_val

    def one_product_3call(p):
        """plan -> symbolic (row pointer, nnz(C) read back) -> numeric."""
        plan = binding.spgemm_plan(p["dA"], p["dB"], p["ws"], None, stream)
        try:
            nnz = binding.spgemm_symbolic(plan, p["C_rp"], stream)
            C_col = torch.empty(nnz, dtype=torch.int32, device=dev)
            C_val = torch.empty(nnz, dtype=torch.float64, device=dev)
            binding.spgemm_numeric(plan, p["dA"].val, p["dB"].val, C_col, C_val, stream)
        finally:
            binding.spgemm_free(plan)

    def step(record=False):
        for p in prods:
            one_product(p, record)

    for _ in range(max(args.warmup, 3)):
        step()
    # the kernel-timing events of the timed steps, created (first record) before the timed region
    for p in prods:
        p["ev_free"] = []
        for _ in range(args.steps):
            pair = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for ev in pair:
                ev.record(stream)
            p["ev_free"].append(pair)
    torch.cuda.synchronize()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    with ClockSampler(local_rank) as clk:
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step(record=True)
        t1.record(stream)
        barrier()
    ms = ranks.max_over_ranks(t0.elapsed_time(t1) / args.steps, dist, dev)
    # the last timed step's C, kept for the full-size check against the oracle (after all timing)
    if rank == 0 and world == 1 and not args.no_parity:
        for p in prods:
            C_col, C_val = p["last_C"]
            nnz = p["nnz"]
            p["C_host"] = (p["C_rp"].cpu().numpy().astype(np.int64), C_col[:nnz].cpu().numpy(),
                           C_val[:nnz].cpu().numpy())
    for p in prods:
        p.pop("last_C", None)

    # the three-call path (plan / symbolic / numeric) on the same inputs, for comparison
    for _ in range(2):
        for p in prods:
            one_product_3call(p)
    torch.cuda.synchronize()
    a3, b3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a3.record(stream)
    for _ in range(args.steps):
        for p in prods:
            one_product_3call(p)
    b3.record(stream)
    torch.cuda.synchronize()
    ms_3call = a3.elapsed_time(b3) / args.steps

    # numeric-only (pattern reuse): values recomputed on a planned structure, by the numeric pass
    # and by the replay of a recorded position map
    numeric_only = run_numeric_only(args, prods, dev, stream, binding, torch)

    F_total = sum(p["info"]["products"] for p in prods)
    flop_step = 2 * F_total
    value = world * flop_step / (ms * 1e-3) / 1e9
    bw, bw_kind = hbm_peak()
    detail = {}
    bytes_step = 0
    dominant = None
    for p in prods:
        bmin = roofline.bytes_min(p["A"], p["B"], p["nnz"])
        bytes_step += bmin
        num_ms = float(np.mean([a.elapsed_time(b) for a, b in zip(p["ev0"], p["ev1"])]))
        cls = p["info"]["rows_per_class"]
        wide = p["info"]["max_row_products"] > 32 and cls["M2"] > 0
        # default options: 32-product tiles use the direct form, 64-product rows the four-lanes-per-row form;
        # longer rows add the warp-, block- and dense-class kernels to the same call
        kern = "k_merge_quad<fused>" if wide else "k_merge<fused,32>"
        if any(cls[c] > 0 for c in ("W", "B", "G")):
            kern = "spgemm_compute (" + kern + " + " + ", ".join(c for c in ("W", "B", "G") if cls[c] > 0) + " class kernels)"
        d = {"F": p["info"]["products"], "nnz_c": p["nnz"], "bytes_min": bmin, "compute_ms": num_ms,
             "compute_kernel": kern, "rows_per_class": cls,
             "compute_gbs": bmin / (num_ms * 1e-3) / 1e9,
             "compute_gflops": 2 * p["info"]["products"] / (num_ms * 1e-3) / 1e9}
        detail[p["name"]] = d
        if dominant is None or num_ms > detail[dominant]["compute_ms"]:
            dominant = p["name"]
    dom = detail[dominant]
    achieved = dom["compute_gbs"]
    roof = {"bound": "hbm", "achieved": achieved, "peak": bw, "unit": "GB/s", "frac": achieved / bw,
            "traffic": committed_traffic(dom["compute_kernel"]), "kernel": dom["compute_kernel"],
            "workload": dominant, "peak_kind": f"{bw_kind} (MEASURED_PEAKS.json hbm_gbs)",
            "step_frac_of_hbm_roofline": bytes_step / (ms * 1e-3) / 1e9 / bw,
            "algorithmic_bytes": "read A (4(m+1)+12nnzA) + each referenced B row once + write C (4(m+1)+12nnzC)"}
    launches_per_step = 0
    for p in prods:
        cls = p["info"]["rows_per_class"]
        others = sum(1 for c in ("W", "B", "G") if cls[c] > 0)
        launches_per_step += 1 + 1 + 2 * others   # bin, fused merge pass, symbolic + numeric per other class

    # end to end through the C ABI from pinned host buffers
    e2e = run_e2e(args, prods, dev, stream, binding, torch, world, dist)

    cpu = cpu_combined = cpu_all = parity = None
    if rank == 0 and world == 1:
        workers = max(1, min(os.cpu_count() or 1, 64))
        cpu = oracle_protocol(work, 1.0 / 64)
        try:
            cpu_all = oracle_all_cores(args.workload, work, workers)
        except Exception as e:  # noqa: BLE001 -- a baseline must not cost the GPU measurement
            cpu_all = {"unavailable": f"{type(e).__name__}: {e}"}
        cpu_combined = combined_baseline(work)
        if not args.no_parity:
            try:
                parity = check_full_products(args.workload, [(p["name"], p["C_host"][0], p["C_host"][1],
                                                              p["C_host"][2]) for p in prods], workers)
            except Exception as e:  # noqa: BLE001
                parity = {"unavailable": f"{type(e).__name__}: {e}"}

    extras = {}
    if not args.no_extras and args.workload == "plain":
        extras["batched"] = run_batched(args, dev, binding, torch)
        extras["backward"] = run_backward(args, dev, binding, torch)
        extras["long_rows"] = run_long_rows(args, dev, binding, torch)

    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.workload == "plain" else args.workload, "indices": "int32", "values": "float64",
                       "l2": "inputs (~2.5 GB per step) larger than L2; no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
            "cpu_baseline_combined": cpu_combined, "parity_full_size": parity, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk.summary(), "detail": detail,
            "three_call": {"ms_per_step": ms_3call, "value": world * flop_step / (ms_3call * 1e-3) / 1e9,
                           "path": "plan / symbolic / numeric"},
            "numeric_only": numeric_only,
            "path": "plan (binning, F read back) + single-pass compute (nnz(C) read back)",
            **extras}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_e2e(args, prods, dev, stream, binding, torch, world, dist=None):
    """Same metric through the C ABI with host buffers: H2D of A, B and D2H of C inside the timed region."""
    host = []
    h2d = d2h = 0
    for p in prods:
        A, B = p["A"], p["B"]
        hA = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (A.row_ptr, A.col_idx, A.val)]
        hB = hA if B is A else [torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
                                for x in (B.row_ptr, B.col_idx, B.val)]
        dA = binding.DeviceCSR(A.rows, A.cols, *[torch.empty_like(t, device=dev) for t in hA])
        dB = dA if B is A else binding.DeviceCSR(B.rows, B.cols, *[torch.empty_like(t, device=dev) for t in hB])
        nnz = p["nnz"]
        outs = [torch.empty(A.rows + 1, dtype=torch.int32).pin_memory(),
                torch.empty(nnz, dtype=torch.int32).pin_memory(), torch.empty(nnz, dtype=torch.float64).pin_memory()]
        host.append((p, hA, hB, dA, dB, outs))
        h2d += sum(t.numel() * t.element_size() for t in hA)
        if B is not A:
            h2d += sum(t.numel() * t.element_size() for t in hB)
        d2h += sum(t.numel() * t.element_size() for t in outs)

    # Copies on their own streams: both products' inputs go first, and product i's result comes
    # back while product i+1 -- or the next step's first product -- is copied in, planned and
    # computed (the plan and compute calls synchronise only the compute stream).  Every step still
    # copies its own inputs in and its own result out; the timed loop ends with a full synchronise.
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def e2e_step():
        ev_in = []
        for p, hA, hB, dA, dB, outs in host:
            with torch.cuda.stream(s_in):
                for d, h in zip((dA.row_ptr, dA.col_idx, dA.val), hA):
                    d.copy_(h, non_blocking=True)
                if dB is not dA:
                    for d, h in zip((dB.row_ptr, dB.col_idx, dB.val), hB):
                        d.copy_(h, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s_in)
            ev_in.append(ev)
        keep = []
        for (p, hA, hB, dA, dB, outs), ev in zip(host, ev_in):
            stream.wait_event(ev)
            plan = binding.spgemm_plan(dA, dB, p["ws"], None, stream)
            try:
                F = binding.spgemm_plan_info(plan)["products"]
                # C of this step: its own buffers, still being copied out while the next step runs
                C_rp = torch.empty(dA.rows + 1, dtype=torch.int32, device=dev)
                C_col = torch.empty(max(F, 1), dtype=torch.int32, device=dev)
                C_val = torch.empty(max(F, 1), dtype=torch.float64, device=dev)
                nnz = binding.spgemm_compute(plan, dA.val, dB.val, C_rp, C_col, C_val, stream)
            finally:
                binding.spgemm_free(plan)
            done = torch.cuda.Event()
            done.record(stream)
            s_out.wait_event(done)
            with torch.cuda.stream(s_out):
                outs[0].copy_(C_rp, non_blocking=True)
                outs[1].copy_(C_col[:nnz], non_blocking=True)
                outs[2].copy_(C_val[:nnz], non_blocking=True)
            for t in (C_rp, C_col, C_val):
                t.record_stream(s_out)
            keep.append((C_rp, C_col, C_val))
        # the next step's input copies may overwrite A and B only after this step's computes,
        # which the compute calls have already waited for

    steps = max(3, min(args.steps, 10))
    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        e2e_step()
    torch.cuda.synchronize()
    from paper_1303_1651_gb300 import ranks
    dt = ranks.max_over_ranks((time.perf_counter() - t0) / steps, dist, dev)
    F_total = sum(p["info"]["products"] for p in prods)
    return {"value": world * 2 * F_total / dt / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3, "steps": steps}


def run_batched(args, dev, binding, torch):
    """512 independent products (half Laplacian^2, half random*random, N log-uniform 256..65536):
    one graph-replayed batch against the per-matrix loop, default and autotuned row classes."""
    from paper_1303_1651_gb300 import batched, tune
    probs = synth.batch_problems(count=512, seed=synth.SEED_BATCH)
    A, B, lay = batched.concat(probs)
    dA, dB = binding.DeviceCSR.from_host(A, dev), binding.DeviceCSR.from_host(B, dev)
    F = None
    out = {"problems": len(probs), "rows": A.rows, "nnz_A": A.nnz, "nnz_B": B.nnz}
    steps = max(3, args.steps)

    def time_batch(opt):
        bp = batched.BatchedProduct(dA, dB, opt)
        for _ in range(3):
            bp.run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            bp.run()
        e1.record()
        torch.cuda.synchronize()
        bp.check()
        f = bp.info["products"]
        ms = e0.elapsed_time(e1) / steps
        bp.close()
        return f, ms

    F, ms = time_batch(None)
    out["F"] = F
    out["batched_ms"] = ms
    out["batched_gflops"] = 2 * F / (ms * 1e-3) / 1e9
    tuned = tune.tune(dA, dB, cache_path=None)
    topt = binding.options(**tuned["options"]) if tuned["options"] else None
    _, tms = time_batch(topt)
    out["tuned_options"] = tuned["options"]
    out["tuned_batched_ms"] = tms
    out["tuned_batched_gflops"] = 2 * F / (tms * 1e-3) / 1e9
    devp = [(binding.DeviceCSR.from_host(Ap, dev), binding.DeviceCSR.from_host(Bp, dev)) if Bp is not Ap
            else (lambda d: (d, d))(binding.DeviceCSR.from_host(Ap, dev)) for Ap, Bp in probs]
    pm = batched.PerMatrix(devp, topt)
    pm.run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = max(2, min(steps, 5))
    for _ in range(reps):
        pm.run()
    torch.cuda.synchronize()
    pms = (time.perf_counter() - t0) / reps * 1e3
    out["per_matrix_ms"] = pms
    out["per_matrix_gflops"] = 2 * pm.F / (pms * 1e-3) / 1e9
    out["speedup_batched_vs_per_matrix"] = pms / min(ms, tms)
    del pm
    # (ii) the per-matrix loop without host synchronisation: every problem planned once (untimed),
    # its C sized by its multiplication count, then one spgemm_compute_async per problem
    items = []
    try:
        for dAp, dBp in devp:
            ws = torch.empty(binding.spgemm_workspace_size(dAp, dBp, topt), dtype=torch.uint8, device=dev)
            plan = binding.spgemm_plan(dAp, dBp, ws, topt)
            f = max(binding.spgemm_plan_info(plan)["products"], 1)
            items.append((plan, dAp, dBp, ws, torch.empty(dAp.rows + 1, dtype=torch.int32, device=dev),
                          torch.empty(f, dtype=torch.int32, device=dev), torch.empty(f, dtype=torch.float64, device=dev)))

        def loop():
            for plan, dAp, dBp, _, C_rp, C_col, C_val in items:
                binding.spgemm_compute_async(plan, dAp.val, dBp.val, C_rp, C_col, C_val)

        loop()
        torch.cuda.synchronize()
        for it in items:
            binding.spgemm_status(it[0])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            loop()
        e1.record()
        torch.cuda.synchronize()
        ams = e0.elapsed_time(e1) / reps
    finally:
        for it in items:
            binding.spgemm_free(it[0])
    out["per_matrix_async_ms"] = ams
    out["per_matrix_async_gflops"] = 2 * F / (ams * 1e-3) / 1e9
    out["per_matrix_async_note"] = "planned beforehand (untimed); one spgemm_compute_async per problem, no host syncs"
    out["speedup_batched_vs_per_matrix_async"] = ams / min(ms, tms)
    return out


def run_long_rows(args, dev, binding, torch):
    """The paper's 0.1 % fill workload (Section IV-B): random N x N with round(0.001 N) entries per
    row, so a row of C gathers about (0.001 N)^2 products.  Per N: plan + single-pass compute under
    the default classes and under each class forced (warp W, block B, dense G, where the rows fit
    it), and, for the warp class, its orderings forced (bit vector over [min, max] = the MinMax
    store, register sort = the Sort store, hash).  GFLOP/s and fraction of the HBM roofline."""
    bw, _ = hbm_peak()
    steps = max(3, min(args.steps, 10))
    off = dict(m1_max_u=-1, m2_max_u=-1)
    offw = dict(off, warp_max_u=1024)
    variants = [("default", {}), ("W", offw), ("B", dict(off, warp_max_u=-1)),
                ("G", dict(off, warp_max_u=-1, block_max_u=-1)),
                ("W-minmax", dict(offw, warp_order=1)), ("W-sort", dict(offw, warp_order=2)),
                ("W-hash", dict(offw, warp_order=3))]
    out = {"fill": 0.001, "points": []}
    for N in (5000, 10000, 20000, 30000, 38000, 50000, 70000):
        A = synth.random_fill(N, 0.001, synth.SEED_A + N)
        B = synth.random_fill(N, 0.001, synth.SEED_B + N)
        dA, dB = binding.DeviceCSR.from_host(A, dev), binding.DeviceCSR.from_host(B, dev)
        k = int(A.row_ptr[1])
        pt = {"N": N, "k": k, "products_per_row": k * k, "by_class": {}}
        for name, o in variants:
            if name.startswith("W") and k * k > 1024:
                continue
            if name == "B" and k * k > 8192:
                continue
            opt = binding.options(**o) if o else None
            ws = torch.empty(binding.spgemm_workspace_size(dA, dB, opt), dtype=torch.uint8, device=dev)

            def step():
                plan = binding.spgemm_plan(dA, dB, ws, opt)
                try:
                    info = binding.spgemm_plan_info(plan)
                    f = max(info["products"], 1)
                    C_col = torch.empty(f, dtype=torch.int32, device=dev)
                    C_val = torch.empty(f, dtype=torch.float64, device=dev)
                    C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
                    return binding.spgemm_compute(plan, dA.val, dB.val, C_rp, C_col, C_val), info
                finally:
                    binding.spgemm_free(plan)

            for _ in range(2):
                nnz, info = step()
            torch.cuda.synchronize()
            ts = []
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                step()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            t = float(np.median(ts))
            bmin = roofline.bytes_min(A, B, nnz)
            pt["by_class"][name] = {"ms": t, "gflops": 2 * info["products"] / (t * 1e-3) / 1e9,
                                    "frac_hbm": bmin / (t * 1e-3) / 1e9 / bw,
                                    "rows_per_class": info["rows_per_class"]}
            pt["nnz_c_per_row"] = nnz / N
        forced = {c: v["ms"] for c, v in pt["by_class"].items() if c in ("W", "B", "G")}
        pt["fastest_class"] = min(forced, key=forced.get)
        orders = {c: v["ms"] for c, v in pt["by_class"].items() if c.startswith("W-")}
        if orders:
            pt["fastest_warp_ordering"] = min(orders, key=orders.get)
        out["points"].append(pt)
        del dA, dB
        torch.cuda.empty_cache()
    return out


def run_backward(args, dev, binding, torch):
    """C = A*B with A random 262144 x 262144 (16 per row), B the 512 x 512 grid Laplacian;
    loss = sum(W * C), W ~ N(0, 1) on C's structure: forward + backward (dA and dB)."""
    A = synth.random_k(262144, 16, synth.SEED_A)
    B = synth.laplacian5(512)
    dA, dB = binding.DeviceCSR.from_host(A, dev), binding.DeviceCSR.from_host(B, dev)
    ws = torch.empty(binding.spgemm_workspace_size(dA, dB), dtype=torch.uint8, device=dev)
    tws = torch.empty(binding.spgemm_backward_workspace_size(dA, dB), dtype=torch.uint8, device=dev)
    plan = binding.spgemm_plan(dA, dB, ws)
    try:
        F = binding.spgemm_plan_info(plan)["products"]
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
        C_col = torch.empty(F, dtype=torch.int32, device=dev)
        C_val = torch.empty(F, dtype=torch.float64, device=dev)
        nnz = binding.spgemm_compute(plan, dA.val, dB.val, C_rp, C_col, C_val)
        gen = torch.Generator(device=dev).manual_seed(synth.SEED_W)
        W = torch.randn(nnz, dtype=torch.float64, device=dev, generator=gen)
        gA = torch.empty(A.nnz, dtype=torch.float64, device=dev)
        gB = torch.empty(B.nnz, dtype=torch.float64, device=dev)
        steps = max(3, args.steps)
        for _ in range(2):
            binding.spgemm_backward(plan, dA.val, dB.val, W, gA, gB, tws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            binding.spgemm_backward(plan, dA.val, dB.val, W, gA, gB, tws)
        e1.record()
        torch.cuda.synchronize()
        binding.spgemm_status(plan)
        bms = e0.elapsed_time(e1) / steps
        # forward (plan + compute, host syncs included)
        f0 = time.perf_counter()
        for _ in range(steps):
            p2 = binding.spgemm_plan(dA, dB, ws)
            binding.spgemm_compute(p2, dA.val, dB.val, C_rp, C_col, C_val)
            binding.spgemm_free(p2)
        fms = (time.perf_counter() - f0) / steps * 1e3
    finally:
        binding.spgemm_free(plan)
    return {"F": F, "nnz_c": nnz, "backward_ms": bms, "backward_gflops": 4 * F / (bms * 1e-3) / 1e9,
            "forward_ms": fms, "forward_gflops": 2 * F / (fms * 1e-3) / 1e9,
            "flops_note": "backward does F multiply-adds for dA and F for dB: 4F flops"}


def run_sweep(args):
    """The size sweep on one GPU: per point, plan + single-pass compute (the timed step of the main
    workload), the L2 flushed before every timed step, times from CUDA events per step."""
    import torch
    from paper_1303_1651_gb300 import binding, build
    build.build()
    binding.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    bw, bw_kind = hbm_peak()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)    # larger than L2
    K, W = args.steps, max(args.warmup, 3)
    points = []
    with ClockSampler(0) as clk:
        for N, kind in synth.sweep_points():
            A, B = synth.sweep_problem(N, kind)
            dA = binding.DeviceCSR.from_host(A, dev)
            dB = dA if B is A else binding.DeviceCSR.from_host(B, dev)
            ws = torch.empty(binding.spgemm_workspace_size(dA, dB), dtype=torch.uint8, device=dev)
            C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
            pt = {"N": N, "kind": kind, "rows": A.rows, "nnz_a": A.nnz}
            # nnz(C) and the overflow check from the three-call path, untimed
            plan = binding.spgemm_plan(dA, dB, ws, None, stream)
            try:
                pt["F"] = binding.spgemm_plan_info(plan)["products"]
                pt["nnz_c"] = binding.spgemm_symbolic(plan, C_rp, stream)
            except binding.SpgemmError as e:
                pt["error"] = e.name
            finally:
                binding.spgemm_free(plan)
            if "error" in pt:
                points.append(pt)
                continue
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2 * K)]
            for e in ev:
                for x in e:
                    x.record(stream)

            def step(kev=None):
                plan = binding.spgemm_plan(dA, dB, ws, None, stream)
                try:
                    F = binding.spgemm_plan_info(plan)["products"]
                    C_col = torch.empty(max(F, 1), dtype=torch.int32, device=dev)
                    C_val = torch.empty(max(F, 1), dtype=torch.float64, device=dev)
                    if kev:
                        binding.spgemm_plan_set_events(plan, *kev)
                    return binding.spgemm_compute(plan, dA.val, dB.val, C_rp, C_col, C_val, stream)
                finally:
                    binding.spgemm_free(plan)

            for _ in range(W):
                step()
            step_ms, kern_ms = [], []
            i_clk = len(clk.lines)
            for i in range(K):
                flush.zero_()
                e0, e1 = ev[2 * i]
                e0.record(stream)
                nnz = step(ev[2 * i + 1])
                e1.record(stream)
                torch.cuda.synchronize()
                step_ms.append(e0.elapsed_time(e1))
                kern_ms.append(ev[2 * i + 1][0].elapsed_time(ev[2 * i + 1][1]))
            assert nnz == pt["nnz_c"]
            # the same product through spgemm_multiply: one call, one read-back, C preallocated with
            # capacity F (a caller that reuses its buffers)
            cap = max(pt["F"], 1)
            oC_col = torch.empty(cap, dtype=torch.int32, device=dev)
            oC_val = torch.empty(cap, dtype=torch.float64, device=dev)
            for _ in range(W):
                binding.spgemm_multiply(dA, dB, C_rp, oC_col, oC_val, ws, None, stream)
            one_ms = []
            for i in range(K):
                flush.zero_()
                e0, e1 = ev[2 * i]
                e0.record(stream)
                onnz, _ = binding.spgemm_multiply(dA, dB, C_rp, oC_col, oC_val, ws, None, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                one_ms.append(e0.elapsed_time(e1))
            assert onnz == pt["nnz_c"]
            del oC_col, oC_val
            # the same product as a CUDA graph of spgemm_multiply_async, replayed: the step is the
            # replay and the read-back of nnz(C) (graph_ms), or the replay alone (graph_device_ms)
            gp = binding.GraphProduct(dA, dB, cap)
            for _ in range(W):
                gp.run()
            g_ms, gd_ms = [], []
            for i in range(K):
                flush.zero_()
                e0, e1 = ev[2 * i]
                d0, d1 = ev[2 * i + 1]
                torch.cuda.synchronize()
                e0.record(stream)
                d0.record(stream)
                gp.graph.replay()
                d1.record(stream)
                gnnz, _ = binding.spgemm_multiply_result(gp.ws, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                g_ms.append(e0.elapsed_time(e1))
                gd_ms.append(d0.elapsed_time(d1))
            assert gnnz == pt["nnz_c"]
            del gp
            pt.update({"graph_ms": float(np.median(g_ms)), "graph_device_ms": float(np.median(gd_ms))})
            bmin = roofline.bytes_min(A, B, nnz)
            ms, kms = float(np.median(step_ms)), float(np.median(kern_ms))
            oms = float(np.median(one_ms))
            pt.update({"one_sync_ms": oms, "one_sync_gflops": 2 * pt["F"] / (oms * 1e-3) / 1e9})
            pt.update({"ms": ms, "gflops": 2 * pt["F"] / (ms * 1e-3) / 1e9, "bytes_min": bmin,
                       "frac": bmin / (ms * 1e-3) / 1e9 / bw, "kernel_ms": kms,
                       "kernel_gflops": 2 * pt["F"] / (kms * 1e-3) / 1e9,
                       "kernel_frac": bmin / (kms * 1e-3) / 1e9 / bw,
                       "steps_ms": [round(x, 4) for x in step_ms], "sm_mhz": clk.sm_median(i_clk)})
            points.append(pt)
            if args.verbose:
                print(json.dumps(pt), file=sys.stderr, flush=True)
            del dA, dB, ws, C_rp, A, B
            torch.cuda.empty_cache()
    line = {"metric": METRIC, "mode": "sweep", "unit": "GFLOP/s", "n_gpus": 1, "steps": K, "warmup": W,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "size sweep: N = round(10^(3+i/3)), i = 0..12; Laplacian^2 on a round(sqrt N)^2 "
                                   "grid and random*random with 4, 8, 16 distinct columns per row",
                       "l2": "512 MB buffer written before every timed step",
                       "step": "plan (binning, F read back) + single-pass compute (nnz(C) read back)",
                       "one_sync": "spgemm_multiply: binning and single-pass compute in one call, one read-back, "
                                   "C preallocated with capacity F",
                       "graph": "spgemm_multiply_async captured once in a CUDA graph: graph_ms = replay + "
                                "read-back of nnz(C) (spgemm_multiply_result), graph_device_ms = the replay alone",
                       "kernel": "the compute call's kernels alone (events around them)"},
            "peak": {"hbm_gbs": bw, "kind": f"{bw_kind} (MEASURED_PEAKS.json hbm_gbs)"},
            "clocks": clk.summary(), "points": points}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if args.gpus == 1 else 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.sweep:
        run_sweep(args)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
