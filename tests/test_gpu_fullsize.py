"""Full-size products of the benchmark workload, in the launch configuration bench.py times
(default options), compared with the oracle over every entry (the oracle needs seconds here)."""
import pytest

import oracle
from paper_1303_1651_gb300 import synth
from tests.gpu_util import compare, gpu_product

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fused", [True, False], ids=["fused", "3call"])
def test_laplacian_2048_squared_full(fused):
    A = synth.laplacian5(2048)
    C = gpu_product(A, A, fused=fused)
    assert C["nnz"] == 54484996 and C["info"]["products"] == 104783880
    compare(C, oracle.spgemm(A, A), exact=True)


@pytest.mark.parametrize("fused", [True, False], ids=["fused", "3call"])
def test_random_1M_k8_full(fused):
    A = synth.random_k(1_000_000, 8, synth.SEED_A)
    B = synth.random_k(1_000_000, 8, synth.SEED_B)
    C = gpu_product(A, B, fused=fused)
    assert C["info"]["products"] == 64_000_000
    compare(C, oracle.spgemm(A, B), single=True)
