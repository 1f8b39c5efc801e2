"""Host-side pieces of bench.py, on the CPU: the reference arm's JSON line (the oracle timed on a
row sample), the code hash that keys the stored DRAM traffic (comments must not change it, code
must), and the CPU-baseline helpers."""
import importlib.util
import json
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1303_1651_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "medium",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == "GFLOP/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["n_gpus"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_kernel_hash_ignores_comments_only(tmp_path):
    bench = load_bench()
    ref = bench.kernel_source_hash()
    csrc = tmp_path / "paper_1303_1651_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("common.cuh", "merge.cu"):
        shutil.copy(os.path.join(ROOT, "paper_1303_1651_gb300", "csrc", f), csrc / f)
    (tmp_path / "profiles").mkdir()
    stored = {"k": {"dram_bytes_per_launch": 123, "source_hash": ref}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(stored))
    bench.ROOT = str(tmp_path)
    assert bench.kernel_source_hash() == ref
    assert bench.committed_traffic("k") == 123 and bench.committed_traffic("other") is None
    merge = csrc / "merge.cu"
    text = merge.read_text()
    merge.write_text("// a new comment\n\n" + text.replace("\n", "   // trailing note\n", 3) + "\n\n")
    assert bench.kernel_source_hash() == ref, "a comment changed the hash"
    merge.write_text(text.replace("constexpr int IB = 6;", "constexpr int IB = 7;", 1))
    assert bench.kernel_source_hash() != ref, "a code change kept the hash"
    assert bench.committed_traffic("k") is None


def test_cpu_baseline_helpers():
    bench = load_bench()
    A = synth.random_k(3000, 6, 5)
    B = synth.random_k(3000, 6, 6)
    S = bench.row_sample(A, 0.25)
    assert S.rows == 750 and np.array_equal(S.row_ptr, A.row_ptr[:751])
    assert np.array_equal(S.col_idx, A.col_idx[:S.row_ptr[-1]])
    work = [("r", A, B), ("l", synth.laplacian5(30), None)]
    work[1] = ("l", work[1][1], work[1][1])
    rate, dt, F = bench.combined_rate(work, threads=2)
    assert rate > 0 and dt > 0 and F == oracle.spgemm(A, B)["F"] + oracle.spgemm(work[1][1], work[1][1])["F"]
    rate, dt, F = bench.oracle_rate(work, 0.5)
    assert rate > 0 and F == oracle.spgemm(bench.row_sample(A, 0.5), B)["F"] + \
        oracle.spgemm(bench.row_sample(work[1][1], 0.5), work[1][1])["F"]


def test_combined_baseline_entry(monkeypatch):
    bench = load_bench()
    work = [("r", synth.random_k(4000, 8, 7), synth.random_k(4000, 8, 8))]
    line = bench.combined_baseline(work)
    assert line["value"] > 0 and line["cores"] >= 1 and line["single_thread"]["cores"] == 1
    import baseline

    def broken(*a, **k):
        raise OSError("no C++ compiler")
    monkeypatch.setattr(baseline, "combined", broken)
    assert bench.combined_baseline(work) == {"unavailable": "OSError: no C++ compiler"}


def test_oracle_protocol_and_all_cores():
    import bench
    work = bench.make_workload("small")
    line = bench.oracle_protocol(work, 0.25, min_s=0.2, min_runs=3)
    assert line["runs"] >= 3 and line["value"] >= line["median"] > 0
    assert line["cores"] == line["threads"] == 1 and line["cpu_model"]
    allc = bench.oracle_all_cores("small", work, workers=2, min_s=0.2, min_runs=2)
    assert allc["cores"] == 2 and allc["runs"] >= 2 and allc["value"] > 0


def test_full_size_check_against_the_oracle():
    import bench
    work = bench.make_workload("small")
    results = []
    for name, A, B in work:
        R = oracle.spgemm(A, B)
        results.append((name, R["row_ptr"], R["col_idx"], R["val"].copy()))
    out = bench.check_full_products("small", results, workers=2)
    for name, _, col, _ in results:
        v = out[name]
        assert v["pattern_equal"] and v["max_err_over_sum_abs"] == 0 and v["max_plain_rel_err"] == 0
        assert v["entries"] == col.size
    # a planted value error shows in both measures; a planted column error in the pattern check
    name, rp, col, val = results[1]
    val[123] *= 1 + 1e-9
    out = bench.check_full_products("small", [(name, rp, col, val)], workers=2)[name]
    assert out["pattern_equal"] and 1e-10 < out["max_plain_rel_err"] < 1e-8 and out["max_err_over_sum_abs"] > 1e-10
    col = col.copy()
    col[5], col[6] = col[6], col[5]
    assert not bench.check_full_products("small", [(name, rp, col, val)], workers=2)[name]["pattern_equal"]
