"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Pattern (row_ptr, col_idx) must match bit-exactly; values within 1e-12 of the
sum of |a*b| of the entry.  Merge-class rows sum in the oracle's order, so
their values are also compared bit-exactly."""
import numpy as np
import pytest

import oracle
from paper_1303_1651_gb300 import synth
from tests.gpu_util import compare, gpu_product

pytestmark = pytest.mark.gpu

PATHS = pytest.mark.parametrize("fused", [False, True], ids=["3call", "fused"])


def opts(**kw):
    from paper_1303_1651_gb300 import binding
    return binding.options(**kw)


@PATHS
def test_laplacian_64_squared(fused):
    A = synth.laplacian5(64)
    C = gpu_product(A, A, fused=fused)
    R = oracle.spgemm(A, A)
    compare(C, R, exact=True)
    assert C["info"]["products"] == 100104 and C["nnz"] == 51972


@PATHS
def test_random_4096_k8(fused):
    A, B = synth.random_k(4096, 8, synth.SEED_A), synth.random_k(4096, 8, synth.SEED_B)
    compare(gpu_product(A, B, fused=fused), oracle.spgemm(A, B), single=True)


@PATHS
@pytest.mark.parametrize("k", [1, 2, 4, 5, 7, 8])
def test_random_merge_classes(k, fused):
    A, B = synth.random_k(3000, k, 11 + k), synth.random_k(3000, k, 31 + k)
    C = gpu_product(A, B, fused=fused)
    compare(C, oracle.spgemm(A, B), single=True)


@PATHS
@pytest.mark.parametrize("k", [9, 16, 32])
def test_random_hash_classes(k, fused):
    A, B = synth.random_k(2000, k, 5 + k), synth.random_k(2000, k, 7 + k)
    C = gpu_product(A, B, fused=fused)
    compare(C, oracle.spgemm(A, B))
    assert C["info"]["rows_per_class"]["W"] + C["info"]["rows_per_class"]["B"] > 0


@PATHS
def test_power_law_all_classes(fused):
    A = synth.power_law(3000, 3000, 3, alpha=1.5, max_len=3000)
    B = synth.power_law(3000, 4000, 4, alpha=1.5, max_len=400)
    C = gpu_product(A, B, fused=fused)
    R = oracle.spgemm(A, B)
    compare(C, R)
    cls = C["info"]["rows_per_class"]
    assert all(cls[c] > 0 for c in ("M1", "M2", "W", "B", "G")), cls


@pytest.mark.parametrize("forced", [
    dict(m1_max_u=-1, m2_max_u=-1),                                   # everything hashed
    dict(m1_max_u=-1, m2_max_u=-1, warp_max_u=-1),                    # block hash
    dict(m1_max_u=-1, m2_max_u=-1, warp_max_u=-1, block_max_u=-1),   # dense fallback only
    dict(m1_max_u=4, m2_max_u=16, warp_max_u=40, block_max_u=100, dense_slabs=3),
])
@PATHS
def test_forced_classes(forced, fused):
    A = synth.power_law(1500, 1200, 8, alpha=1.7, max_len=300)
    B = synth.power_law(1200, 900, 9, alpha=1.7, max_len=100)
    compare(gpu_product(A, B, opts(**forced), fused=fused), oracle.spgemm(A, B))


@PATHS
def test_laplacian_forced_classes_exact(fused):
    A = synth.laplacian5(40)
    R = oracle.spgemm(A, A)
    for forced in (dict(m1_max_u=-1, m2_max_u=-1), dict(m1_max_u=-1, m2_max_u=-1, warp_max_u=-1, block_max_u=-1)):
        compare(gpu_product(A, A, opts(**forced), fused=fused), R, exact=True)   # small integers: every order is exact


@PATHS
def test_rectangular_and_empty_rows(fused):
    rng = np.random.default_rng(12)
    lengths = rng.integers(0, 20, size=700)
    lengths[100:200] = 0                        # a block of empty rows
    A = synth.random_lengths(lengths, 300, 12)  # 700 x 300
    blen = rng.integers(0, 25, size=300)
    blen[::7] = 0                               # empty rows of B as well
    B = synth.random_lengths(blen, 1100, 13)    # 300 x 1100
    compare(gpu_product(A, B, fused=fused), oracle.spgemm(A, B))


@PATHS
def test_degenerate_shapes(fused):
    one = synth.from_dense(np.array([[2.5]]))
    C = gpu_product(one, one, fused=fused)
    assert list(C["val"]) == [6.25]
    Z = synth.CSR(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = synth.random_k(5, 2, 1)
    C = gpu_product(Z, B, fused=fused)
    assert C["nnz"] == 0 and list(C["row_ptr"]) == [0]
    E = synth.CSR(4, 5, np.zeros(5, np.int32), np.zeros(0, np.int32), np.zeros(0))
    C = gpu_product(E, B, fused=fused)
    assert C["nnz"] == 0 and list(C["row_ptr"]) == [0] * 5
    Bz = synth.CSR(5, 3, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0))
    A = synth.random_k(7, 2, 3, ncols=5)
    C = gpu_product(A, Bz, fused=fused)      # every B row empty
    assert C["nnz"] == 0


@PATHS
def test_cancellation_and_explicit_zeros(fused):
    A = synth.CSR(1, 2, np.array([0, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, 1.0]))
    B = synth.CSR(2, 1, np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([1.0, -1.0]))
    C = gpu_product(A, B, fused=fused)
    assert C["nnz"] == 1 and C["val"][0] == 0.0
    Az = synth.random_k(500, 6, 3)
    Az.val[::3] = 0.0
    Bz = synth.random_k(500, 6, 4)
    Bz.val[::5] = 0.0
    compare(gpu_product(Az, Bz, fused=fused), oracle.spgemm(Az, Bz), single=True)


@PATHS
def test_unsorted_A_and_duplicates_in_A(fused):
    A = synth.duplicate_entries(synth.random_k(800, 5, 21), 22)   # unsorted rows with repeated columns
    B = synth.random_k(800, 6, 23)
    compare(gpu_product(A, B, fused=fused), oracle.spgemm(A, B))


@PATHS
def test_unsorted_and_duplicate_B_rows(fused):
    # the merge classes sort every product, so B's rows may be in any order and repeat columns
    A = synth.random_k(600, 4, 31)
    B = synth.shuffle_rows(synth.random_k(600, 6, 32), 33)
    R = oracle.spgemm(A, B)
    compare(gpu_product(A, B, fused=fused), R, single=True)
    compare(gpu_product(A, B, opts(m1_max_u=-1, m2_max_u=-1), fused=fused), R)
    Bd = synth.duplicate_entries(synth.random_k(600, 5, 34), 35)
    compare(gpu_product(A, Bd, fused=fused), oracle.spgemm(A, Bd), single=True)
    compare(gpu_product(A, Bd, opts(m1_max_u=-1, m2_max_u=-1), fused=fused), oracle.spgemm(A, Bd))


def test_numeric_repeatable_with_new_values():
    from paper_1303_1651_gb300 import binding
    import torch
    A, B = synth.random_k(2000, 7, 41), synth.laplacian5(45)
    A = synth.random_k(2025, 7, 41)
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    prod = binding.Product(dA, dB)
    try:
        for t in range(3):
            A2 = A.copy(); A2.val = A.val * (t + 1) - t
            C = prod.numeric(A_val=torch.from_numpy(A2.val).cuda())
            binding.spgemm_status(prod.plan)
            out = C.to_host()
            compare(out, oracle.spgemm(A2, B), single=True)
    finally:
        prod.close()


def test_validate_option_flags_bad_columns():
    from paper_1303_1651_gb300 import binding
    A = synth.random_k(100, 3, 51)
    B = synth.random_k(100, 3, 52)
    B.col_idx[5] = 1000       # out of range column in B
    with pytest.raises(binding.SpgemmError) as e:
        gpu_product(A, B, opts(validate=1))
    assert e.value.name == "SPGEMM_ERR_INVALID"


def test_fused_capacity_too_small_reported():
    import torch
    from paper_1303_1651_gb300 import binding
    A = synth.random_k(3000, 6, 61)
    B = synth.random_k(3000, 6, 62)
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    ws = torch.empty(binding.spgemm_workspace_size(dA, dB), dtype=torch.uint8, device="cuda")
    plan = binding.spgemm_plan(dA, dB, ws)
    try:
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device="cuda")
        cap = 1000
        C_col = torch.full((cap + 64,), -7, dtype=torch.int32, device="cuda")
        C_val = torch.zeros(cap + 64, dtype=torch.float64, device="cuda")
        with pytest.raises(binding.SpgemmError) as e:
            binding.spgemm_compute(plan, dA.val, dB.val, C_rp, C_col[:cap], C_val[:cap])
        assert e.value.name == "SPGEMM_ERR_OVERFLOW"
        assert bool((C_col[cap:] == -7).all())      # nothing written past the capacity
    finally:
        binding.spgemm_free(plan)


@pytest.mark.parametrize("frac", [0.0, 0.3, 0.7, 0.999])
def test_fused_capacity_too_small_all_classes(frac):
    """A capacity below nnz(C) on a product with rows of every class.  The hash and dense kernels
    write their rows after the fused pass has placed every row, so the row pointer they read must
    stay inside the capacity: OVERFLOW, C_row_ptr within [0, capacity], nothing written past the
    capacity, and a numeric pass on the failed structure refused."""
    import torch
    from paper_1303_1651_gb300 import binding
    A = synth.power_law(3000, 3000, 3, alpha=1.5, max_len=3000)
    B = synth.power_law(3000, 4000, 4, alpha=1.5, max_len=400)
    nnz = int(oracle.spgemm(A, B)["row_ptr"][-1])
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    ws = torch.empty(binding.spgemm_workspace_size(dA, dB), dtype=torch.uint8, device="cuda")
    plan = binding.spgemm_plan(dA, dB, ws)
    try:
        cls = binding.spgemm_plan_info(plan)["rows_per_class"]
        assert all(cls[c] > 0 for c in ("M1", "M2", "W", "B", "G")), cls
        cap = int(frac * nnz)
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device="cuda")
        C_col = torch.full((cap + 4096,), -7, dtype=torch.int32, device="cuda")
        C_val = torch.full((cap + 4096,), 5.0, dtype=torch.float64, device="cuda")
        with pytest.raises(binding.SpgemmError) as e:
            binding.spgemm_compute(plan, dA.val, dB.val, C_rp, C_col[:cap], C_val[:cap])
        assert e.value.name == "SPGEMM_ERR_OVERFLOW"
        assert bool((C_col[cap:] == -7).all()) and bool((C_val[cap:] == 5.0).all())
        rp = C_rp.cpu().numpy()
        assert rp.min() >= 0 and rp.max() <= cap and (np.diff(rp) >= 0).all()
        with pytest.raises(binding.SpgemmError) as e:
            binding.spgemm_numeric(plan, dA.val, dB.val, C_col, C_val)
        assert e.value.name == "SPGEMM_ERR_STATE"
    finally:
        binding.spgemm_free(plan)


def test_fused_then_numeric_with_new_values():
    import torch
    from paper_1303_1651_gb300 import binding
    A = synth.random_k(5000, 7, 71)
    B = synth.laplacian5(70)
    A = synth.random_k(4900, 7, 71)
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    ws = torch.empty(binding.spgemm_workspace_size(dA, dB), dtype=torch.uint8, device="cuda")
    plan = binding.spgemm_plan(dA, dB, ws)
    try:
        F = binding.spgemm_plan_info(plan)["products"]
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device="cuda")
        C_col = torch.empty(F, dtype=torch.int32, device="cuda")
        C_val = torch.empty(F, dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        binding.spgemm_plan_set_events(plan, e0, e1)
        nnz = binding.spgemm_compute(plan, dA.val, dB.val, C_rp, C_col, C_val)
        assert e0.elapsed_time(e1) > 0
        R = oracle.spgemm(A, B)
        got = dict(row_ptr=C_rp.cpu().numpy(), col_idx=C_col[:nnz].cpu().numpy(), val=C_val[:nnz].cpu().numpy())
        compare(got, R, single=True)
        A2 = A.copy(); A2.val = -2.0 * A.val
        binding.spgemm_numeric(plan, torch.from_numpy(A2.val).cuda(), dB.val, C_col, C_val)
        binding.spgemm_status(plan)
        got = dict(row_ptr=C_rp.cpu().numpy(), col_idx=C_col[:nnz].cpu().numpy(), val=C_val[:nnz].cpu().numpy())
        compare(got, oracle.spgemm(A2, B), single=True)
    finally:
        binding.spgemm_free(plan)


@PATHS
@pytest.mark.parametrize("ncols,k", [(2000, 12), (300_000, 12), (300_000, 30), (30_000_000, 10), (16_000_000, 12),
                                     (30_000_000, 12), (6_000_000, 30), (30_000_000, 4)],
                         ids=["bitvector", "regsort-256", "regsort-1024", "regsort-128-range-2^25",
                              "regsort-256-range-2^24", "hash-256", "hash-1024", "hash-16-range-2^25"])
def test_warp_class_orderings(ncols, k, fused):
    # rows of k entries of A times rows of k entries of B: u = k^2 products, warp class W (the
    # sort classes are switched off, so the rows of 16 products go there too); the column range
    # of B picks the ordering (bit vector / register sort / hash table).  The register sort's keys
    # hold the column offset above a 7- to 10-bit product index (by the sort size that holds u),
    # so it takes ranges below 2^25 (u <= 128) down to 2^22 (u <= 1024); past 2^22 only rows of
    # more than 32 products take it.
    A = synth.random_k(700, k, 81, ncols=400)
    B = synth.random_k(400, k, 82, ncols=ncols)
    C = gpu_product(A, B, opts(m1_max_u=-1, m2_max_u=-1, warp_max_u=1024), fused=fused)
    assert C["info"]["rows_per_class"]["W"] == 700
    compare(C, oracle.spgemm(A, B), single=True)


@PATHS
@pytest.mark.parametrize("mode", [1, 2], ids=["values-from-B", "values-staged"])
def test_merge_value_modes(mode, fused):
    # both ways of reading B's values in the sort classes, on short (32) and long (64) tiles
    L = synth.laplacian5(50)
    compare(gpu_product(L, L, opts(merge_values=mode), fused=fused), oracle.spgemm(L, L), exact=True)
    for k in (3, 8):
        A, B = synth.random_k(3000, k, 90 + k, ncols=2500), synth.random_k(2500, k, 91 + k)
        compare(gpu_product(A, B, opts(merge_values=mode), fused=fused), oracle.spgemm(A, B), single=True)
    A = synth.duplicate_entries(synth.random_k(900, 5, 95), 96)
    Bs = synth.shuffle_rows(synth.random_k(900, 6, 97), 98)
    compare(gpu_product(A, Bs, opts(merge_values=mode), fused=fused), oracle.spgemm(A, Bs))


def test_more_live_plans_than_pinned_slots():
    """300 live plans: the first 256 read their counters back through the library's pinned slots,
    the rest through their own copy; both give the oracle's product."""
    from paper_1303_1651_gb300 import binding
    A, B = synth.random_k(200, 3, 97), synth.random_k(200, 3, 98)
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    R = oracle.spgemm(A, B)
    prods = []
    try:
        for _ in range(300):
            prods.append(binding.Product(dA, dB))
        for prod in (prods[0], prods[255], prods[256], prods[299]):
            out = prod.numeric().to_host()
            binding.spgemm_status(prod.plan)
            compare(out, R, single=True)
    finally:
        for prod in prods:
            prod.close()
    # slots come back with the plans
    prod = binding.Product(dA, dB)
    try:
        compare(prod.numeric().to_host(), R, single=True)
    finally:
        prod.close()


@PATHS
@pytest.mark.parametrize("ncols,k", [(9_000_000, 4), (30_000_000, 5), (30_000_000, 8), ((1 << 26) - 2, 6)],
                         ids=["M1-9e6", "M1-3e7", "M2-3e7", "M2-limit"])
def test_sort_classes_wide_b(ncols, k, fused):
    # B wider than 2^23 columns: the sort keys hold the column above the 5- or 6-bit product index
    # only, so the sort classes take every B up to 2^26 - 2 columns
    A = synth.random_k(3000, k, 71, ncols=500)
    B = synth.random_k(500, k, 72, ncols=ncols)
    C = gpu_product(A, B, fused=fused)
    cls = C["info"]["rows_per_class"]
    assert cls["M1"] + cls["M2"] == 3000, cls
    compare(C, oracle.spgemm(A, B), single=True)


@PATHS
def test_sort_classes_off_past_limit(fused):
    # one column more than the keys hold: every row goes to the warp class, same product
    A = synth.random_k(1000, 4, 73, ncols=300)
    B = synth.random_k(300, 4, 74, ncols=(1 << 26) - 1)
    C = gpu_product(A, B, fused=fused)
    cls = C["info"]["rows_per_class"]
    assert cls["M1"] + cls["M2"] == 0 and cls["W"] == 1000, cls
    compare(C, oracle.spgemm(A, B), single=True)


def _groups_across_lanes(case):
    """Rows of up to 64 products whose groups of equal columns cross the lanes of the fused pass
    (four lanes of 16 sorted positions a row): one group of 64, many short groups, groups of 7."""
    rng = np.random.default_rng(620)
    n = 3000
    if case == "one-group-of-64":      # every row of B is one column eight times
        B = synth.CSR(n, n, (np.arange(n + 1) * 8).astype(np.int32), np.full(n * 8, 5, np.int32),
                      rng.uniform(-1, 1, n * 8))
        return synth.random_k(n, 8, 621), B
    if case == "short-groups":         # rows of B with 6..8 entries over 12 columns
        lens = rng.integers(6, 9, n)
        rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
        B = synth.CSR(n, n, rp, rng.integers(0, 12, int(rp[-1])).astype(np.int32), rng.uniform(-1, 1, int(rp[-1])))
        return synth.random_k(n, 8, 622), B
    # seven entries of A times identical rows of nine columns: groups of 7 across 16-position edges
    B = synth.CSR(n, n, (np.arange(n + 1) * 9).astype(np.int32), np.tile(np.arange(100, 109, dtype=np.int32), n),
                  rng.uniform(-1, 1, n * 9))
    return synth.random_k(n, 7, 623), B


@pytest.mark.parametrize("case", ["one-group-of-64", "short-groups", "groups-of-7"])
def test_groups_across_lanes_bit_identical(case):
    # the single pass (four lanes a row) and the three-call path (two lanes a row) sum every group
    # in the same order: C is bit-identical between them, and equal to the oracle
    A, B = _groups_across_lanes(case)
    R = oracle.spgemm(A, B)
    fused = gpu_product(A, B, fused=True)
    three = gpu_product(A, B)
    assert fused["info"]["rows_per_class"]["M2"] > 0
    compare(fused, R, single=True)
    for k in ("row_ptr", "col_idx"):
        assert np.array_equal(np.asarray(fused[k], np.int64), np.asarray(three[k], np.int64))
    assert np.array_equal(np.asarray(fused["val"]).view(np.int64), np.asarray(three["val"]).view(np.int64))
