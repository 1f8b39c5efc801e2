"""Batched form on the GPU: one plan and one CUDA-graph replay for many products."""
import numpy as np
import pytest
import torch

import oracle
from paper_1303_1651_gb300 import batched, binding, synth
from tests.gpu_util import compare
from tests.test_batched_host import small_batch

pytestmark = pytest.mark.gpu


def test_batched_graph_matches_oracle_per_problem_and_replays():
    probs = synth.batch_problems(count=40, seed=11, nmin=64, nmax=3000)
    A, B, lay = batched.concat(probs)
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    bp = batched.BatchedProduct(dA, dB)
    bp.run()
    torch.cuda.synchronize()
    bp.check()
    first = bp.result_host()
    for p, (Ap, Bp) in enumerate(probs):
        ref = oracle.spgemm(Ap, Bp)
        got = batched.split(first, lay, p)
        compare(got, ref, single=True)
    # replay: the same pattern, bit for bit; the values again within the bound (rows of the block,
    # hash and dense classes add their products in no fixed order, so a replay may round differently)
    bp.run()
    torch.cuda.synchronize()
    second = bp.result_host()
    for k in ("row_ptr", "col_idx"):
        assert np.array_equal(first[k], second[k])
    for p, (Ap, Bp) in enumerate(probs):
        compare(batched.split(second, lay, p), oracle.spgemm(Ap, Bp), single=True)
    bp.close()


def test_batched_values_change_between_replays():
    probs = small_batch(seed=3, count=10)
    A, B, lay = batched.concat(probs)
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    bp = batched.BatchedProduct(dA, dB)
    dA.val.mul_(-3.0)                       # in place: the graph reads the same buffer
    bp.run()
    torch.cuda.synchronize()
    A2 = A.copy(); A2.val = A.val * -3.0
    compare(bp.result_host(), oracle.spgemm(A2, B), single=True)
    bp.close()


def test_per_matrix_path_matches_batched():
    probs = small_batch(seed=4, count=8)
    devp = [(binding.DeviceCSR.from_host(Ap), binding.DeviceCSR.from_host(Bp)) for Ap, Bp in probs]
    pm = batched.PerMatrix(devp)
    pm.run()
    assert pm.F == sum(oracle.flops(Ap, Bp) for Ap, Bp in probs)


def test_tuned_batch_matches_oracle_per_problem():
    # the autotuner's choice (whatever it is) must leave every problem's product unchanged
    from paper_1303_1651_gb300 import tune
    probs = synth.batch_problems(count=24, seed=12, nmin=64, nmax=4000)
    A, B, lay = batched.concat(probs)
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    tuned = tune.tune(dA, dB, reps=1, cache_path=None)
    assert len(tuned["trials"]) >= len(tune.CANDIDATES)
    opt = binding.options(**tuned["options"]) if tuned["options"] else None
    bp = batched.BatchedProduct(dA, dB, opt)
    bp.run()
    torch.cuda.synchronize()
    bp.check()
    got = bp.result_host()
    for p, (Ap, Bp) in enumerate(probs):
        compare(batched.split(got, lay, p), oracle.spgemm(Ap, Bp), single=True)
    bp.close()


@pytest.mark.parametrize("cand", list(range(16)))
def test_every_tuner_candidate_matches_oracle(cand):
    from paper_1303_1651_gb300 import tune
    if cand >= len(tune.CANDIDATES):
        pytest.skip("fewer candidates")
    probs = small_batch(seed=13, count=12)
    A, B, lay = batched.concat(probs)
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    c = tune.CANDIDATES[cand]
    bp = batched.BatchedProduct(dA, dB, binding.options(**c) if c else None)
    bp.run()
    torch.cuda.synchronize()
    bp.check()
    compare(bp.result_host(), oracle.spgemm(A, B), single=True)
    bp.close()
