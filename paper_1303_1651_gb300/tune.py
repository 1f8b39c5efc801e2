"""Autotuner for the row-class limits (which accumulator each row uses) and tile sizes.

The per-row choice between strategies is the paper's "Combined" kernel idea (Section IV-B: a
cheap per-row decision, tuned by measurement).  Here the choices are the limits of the classes:
the register-sort classes M1/M2 (up to 32 / 64 products, at most merge_max_k entries of A),
the warp and block hash tables, and the dense fallback.  A merge row with more than 32 products
switches the whole matrix to the 64-product sort tiles, so capping M2 at 32 (sending such rows to
the warp hash) is one of the candidates.

tune(A, B) times spgemm_compute_async for each candidate with CUDA events on the device inputs
and returns the fastest option set; results are cached in a JSON file keyed by the GPU name and
a signature of the inputs' shape.
"""
from __future__ import annotations

import json
import os

import torch

from . import binding

# Each candidate belongs to one group of knobs; the best of each group are also tried together.
CANDIDATES = [
    {},                                           # defaults: M1 <= 32, M2 <= 64, W <= 1024, B <= 4096
    # sort classes: tile size and value path
    {"merge_values": 1},                          # direct form (values read from B, C from the reduce)
    {"merge_values": 2},                          # staged form (values copied with the tile)
    {"m2_max_u": 32, "merge_values": 1},          # 32-row tiles only: 33..64-product rows to class W
    {"m2_max_u": 32},
    {"m1_max_u": 16, "m2_max_u": 32},
    {"merge_max_k": 4},
    {"m1_max_u": -1, "m2_max_u": -1},             # no sort classes: every row to the warp and block classes
    # class limits (bins): rows per warp / per block before the dense accumulator
    {"warp_max_u": 128},
    {"warp_max_u": 512},
    {"warp_max_u": 1024},
    {"block_max_u": 2048},
    # class W: the per-row ordering (Section IV-B's "Combined" switch and its alternatives)
    {"warp_bitvec_ratio": 2},                     # the paper's rule: range below twice the row
    {"warp_bitvec_ratio": 32},
    {"warp_order": 2},                            # register sort wherever its keys fit
    {"warp_order": 3},                            # hash table always
]

GROUPS = {
    "sort": ("merge_values", "m1_max_u", "m2_max_u", "merge_max_k"),
    "bins": ("warp_max_u", "block_max_u"),
    "warp": ("warp_bitvec_ratio", "warp_order"),
}


def group_of(c: dict) -> str | None:
    for g, keys in GROUPS.items():
        if c and all(k in keys for k in c):
            return g
    return None

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "spgemm_gb300_tune.json")


def signature(A: binding.DeviceCSR, B: binding.DeviceCSR, info: dict) -> str:
    name = torch.cuda.get_device_name(A.row_ptr.device)
    cls = info["rows_per_class"]
    return (f"{name}|m={A.rows}|k={A.cols}|n={B.cols}|nnzA={A.nnz}|nnzB={B.nnz}|F={info['products']}"
            f"|maxu={info['max_row_products']}|cls={','.join(str(cls[c]) for c in binding.CLASS_NAMES)}")


def _time(A, B, opt_dict, reps: int) -> float:
    opt = binding.options(**opt_dict) if opt_dict else None
    dev = A.row_ptr.device
    ws = torch.empty(binding.spgemm_workspace_size(A, B, opt), dtype=torch.uint8, device=dev)
    plan = binding.spgemm_plan(A, B, ws, opt)
    try:
        F = max(binding.spgemm_plan_info(plan)["products"], 1)
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device=dev)
        C_col = torch.empty(F, dtype=torch.int32, device=dev)
        C_val = torch.empty(F, dtype=torch.float64, device=dev)
        binding.spgemm_compute_async(plan, A.val, B.val, C_rp, C_col, C_val)
        binding.spgemm_status(plan)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            binding.spgemm_compute_async(plan, A.val, B.val, C_rp, C_col, C_val)
        e1.record()
        torch.cuda.synchronize()
        binding.spgemm_status(plan)
        return e0.elapsed_time(e1) / reps
    finally:
        binding.spgemm_free(plan)


def tune(A: binding.DeviceCSR, B: binding.DeviceCSR, candidates=None, reps: int = 3,
         cache_path: str | None = DEFAULT_CACHE, refresh: bool = False) -> dict:
    """Fastest candidate option set for this product: {"options": {...}, "ms": t, "trials": [...]}."""
    candidates = CANDIDATES if candidates is None else candidates
    dev = A.row_ptr.device
    ws = torch.empty(binding.spgemm_workspace_size(A, B), dtype=torch.uint8, device=dev)
    plan = binding.spgemm_plan(A, B, ws)
    info = binding.spgemm_plan_info(plan)
    binding.spgemm_free(plan)
    key = signature(A, B, info)
    cache = load_cache(cache_path)
    if not refresh and key in cache:
        return cache[key]
    trials = []

    def trial(c):
        try:
            trials.append({"options": c, "ms": _time(A, B, c, reps)})
        except binding.SpgemmError as e:
            trials.append({"options": c, "ms": None, "error": e.name})

    for c in candidates:
        trial(c)
    ok = [t for t in trials if t["ms"] is not None]
    base = next((t["ms"] for t in ok if not t["options"]), None)
    # the best candidate of each group that beat the defaults, tried together
    winners = {}
    for t in ok:
        g = group_of(t["options"])
        if g and (base is None or t["ms"] < base) and (g not in winners or t["ms"] < winners[g]["ms"]):
            winners[g] = t
    if len(winners) > 1:
        merged = {}
        for t in winners.values():
            merged.update(t["options"])
        trial(merged)
        ok = [t for t in trials if t["ms"] is not None]
    best = min(ok, key=lambda t: t["ms"])
    result = {"options": best["options"], "ms": best["ms"], "trials": trials}
    if cache_path:
        cache[key] = result
        save_cache(cache_path, cache)
    return result


def load_cache(path: str | None) -> dict:
    if not path or not os.path.exists(path):
        return {}
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
