"""The bench's accounting reproduces the paper's printed model numbers (tests/golden/paper_model.json)."""
import json
import os

import numpy as np

from paper_1303_1651_gb300 import roofline, synth

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_model.json")))


def test_code_balance_and_limits():
    bc = roofline.code_balance_gustavson(G["index_bytes"], G["value_bytes"])
    assert bc == G["inner_loop_code_balance_bytes_per_flop"]
    assert roofline.l1_limit_flops(G["clock_hz"]) / 1e6 == G["l1_limit_mflops"]
    mem = roofline.light_speed(G["peak_gflops"] * 1e9, G["stream_bandwidth_bytes_per_s"], bc) / 1e6
    assert abs(mem - G["memory_limit_mflops"]) / G["memory_limit_mflops"] < 0.02
    # peak: one mul + one add per cycle
    assert 2 * G["clock_hz"] / 1e9 == G["peak_gflops"]


def test_bytes_min_laplacian():
    n = 64
    A = synth.laplacian5(n)
    nnzA = 5 * n * n - 4 * n
    nnzC = 13 * n * n - 20 * n + 4
    m = n * n
    expect = (4 * (m + 1) + 12 * nnzA) + (4 * m + 12 * nnzA) + (4 * (m + 1) + 12 * nnzC)
    assert roofline.bytes_min(A, A, nnzC) == expect
    assert int(roofline.products_per_row(A, A).sum()) == 25 * (n - 2) ** 2 + 64 * (n - 2) + 36
