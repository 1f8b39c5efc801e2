"""Host side of the batched form: the block-diagonal reading, checked with the oracle (no GPU)."""
import numpy as np

import oracle
from paper_1303_1651_gb300 import batched, synth, tune


def small_batch(seed=0, count=12):
    rng = np.random.default_rng(seed)
    probs = []
    for t in range(count):
        if t % 2 == 0:
            A = synth.laplacian5(int(rng.integers(2, 12)))
            probs.append((A, A))
        else:
            N = int(rng.integers(5, 300))
            k = int(rng.integers(1, min(N, 12) + 1))
            probs.append((synth.random_k(N, k, 10 * t + 1), synth.random_k(N, k, 10 * t + 2)))
    return probs


def test_block_diagonal_product_splits_into_the_problems():
    probs = small_batch()
    A, B, lay = batched.concat(probs)
    C = oracle.spgemm(A, B)
    for p, (Ap, Bp) in enumerate(probs):
        got = batched.split(C, lay, p)
        ref = oracle.spgemm(Ap, Bp)
        assert np.array_equal(got["row_ptr"], ref["row_ptr"])
        assert np.array_equal(got["col_idx"], ref["col_idx"])
        assert np.array_equal(got["val"], ref["val"])      # same products in the same order
    assert C["F"] == sum(oracle.flops(Ap, Bp) for Ap, Bp in probs)


def test_batch_problems_generator_shapes():
    probs = synth.batch_problems(count=8, seed=5, nmin=256, nmax=4096)
    assert len(probs) == 8
    for t, (A, B) in enumerate(probs):
        assert A.cols == B.rows and 200 <= A.rows <= 4096
        if t < 4:
            assert B is A and A.row_ptr[-1] == 5 * int(round(A.rows ** 0.5)) ** 2 - 4 * int(round(A.rows ** 0.5))
        else:
            k = np.diff(A.row_ptr)
            assert k.min() == k.max() and 2 <= k[0] <= 32


def test_tune_cache_roundtrip(tmp_path):
    path = str(tmp_path / "c.json")
    assert tune.load_cache(path) == {}
    tune.save_cache(path, {"k": {"options": {"m2_max_u": 32}, "ms": 1.0}})
    assert tune.load_cache(path)["k"]["options"] == {"m2_max_u": 32}
    assert all(isinstance(c, dict) for c in tune.CANDIDATES) and {} in tune.CANDIDATES
