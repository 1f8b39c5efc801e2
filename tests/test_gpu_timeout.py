"""A bounded device wait that runs out, and the host-side fault injections, on the GPU.

The single-pass product places each tile (or group of tiles) of rows by a decoupled look-back over
the ones before it, a wait bounded by a count of re-reads.  With the testing options
debug_drop_tile (a unit that publishes nothing) and debug_spin_limit (a short bound), the
look-backs that reach the dropped unit give up: the call must return SPGEMM_ERR_TIMEOUT, nothing
is written outside the caller's buffers, and the device stays usable (a normal product right after
equals the oracle).  Nothing here faults, traps or hangs the GPU: every wait ends by its bound."""
import pytest
import torch

import oracle
from paper_1303_1651_gb300 import binding, synth
from tests.gpu_util import compare

pytestmark = pytest.mark.gpu


def fused(A, B, opt):
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    ws = torch.empty(binding.spgemm_workspace_size(dA, dB, opt), dtype=torch.uint8, device="cuda")
    plan = binding.spgemm_plan(dA, dB, ws, opt)
    try:
        F = binding.spgemm_plan_info(plan)["products"]
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device="cuda")
        C_col = torch.full((F + 64,), -7, dtype=torch.int32, device="cuda")
        C_val = torch.empty(F + 64, dtype=torch.float64, device="cuda")
        try:
            binding.spgemm_compute(plan, dA.val, dB.val, C_rp, C_col[:F], C_val[:F])
            return None, C_col
        except binding.SpgemmError as e:
            return e.name, C_col
    finally:
        binding.spgemm_free(plan)


@pytest.mark.parametrize("k,form", [(4, {}), (4, dict(merge_values=2)), (8, {})],
                         ids=["128-row-groups", "32-row-tiles", "32-row-groups"])
def test_lookback_gives_up_and_the_device_stays_usable(k, form):
    A, B = synth.random_k(20_000, k, 481), synth.random_k(20_000, k, 482)
    err, C_col = fused(A, B, binding.options(debug_drop_tile=1 + 100, debug_spin_limit=512, **form))
    assert err == "SPGEMM_ERR_TIMEOUT"
    torch.cuda.synchronize()
    assert bool((C_col[-64:] == -7).all()), "written past the capacity"
    # the same product without the dropped unit, on the same device, right after
    err, _ = fused(A, B, binding.options(debug_spin_limit=512, **form))
    assert err is None
    from tests.gpu_util import gpu_product
    compare(gpu_product(A, B, fused=True), oracle.spgemm(A, B), single=True)


def test_fault_injection_from_the_environment(monkeypatch):
    A, B = synth.random_k(3000, 5, 491), synth.random_k(3000, 5, 492)
    dA, dB = binding.DeviceCSR.from_host(A), binding.DeviceCSR.from_host(B)
    ws = torch.empty(binding.spgemm_workspace_size(dA, dB), dtype=torch.uint8, device="cuda")
    monkeypatch.setenv("SPGEMM_FAULT", "alloc")
    with pytest.raises(binding.SpgemmError, match="ALLOC"):
        binding.spgemm_plan(dA, dB, ws)
    monkeypatch.setenv("SPGEMM_FAULT", "nnz_overflow")
    plan = binding.spgemm_plan(dA, dB, ws)
    try:
        F = binding.spgemm_plan_info(plan)["products"]
        C_rp = torch.empty(A.rows + 1, dtype=torch.int32, device="cuda")
        C_col = torch.empty(F, dtype=torch.int32, device="cuda")
        C_val = torch.empty(F, dtype=torch.float64, device="cuda")
        with pytest.raises(binding.SpgemmError, match="OVERFLOW"):
            binding.spgemm_compute(plan, dA.val, dB.val, C_rp, C_col, C_val)
        with pytest.raises(binding.SpgemmError, match="OVERFLOW"):
            binding.spgemm_symbolic(plan, C_rp)
        monkeypatch.delenv("SPGEMM_FAULT")
        nnz = binding.spgemm_compute(plan, dA.val, dB.val, C_rp, C_col, C_val)
        torch.cuda.synchronize()
        got = dict(row_ptr=C_rp.cpu().numpy(), col_idx=C_col[:nnz].cpu().numpy(), val=C_val[:nnz].cpu().numpy())
        compare(got, oracle.spgemm(A, B), single=True)
    finally:
        binding.spgemm_free(plan)
