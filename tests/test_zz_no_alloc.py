"""The allocation-free entry point (esdp_solve_noalloc), for callers that
cannot call cudaMalloc: its output must match the regular esdp_solve on the
same inputs, call after call (the shared device workspace keeps the previous
call's contents, so a second call checks that everything that must start at
zero is cleared), and assets too large for the fixed workspace must be
rejected with a clear error.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2511_15629_b300 import build as B
from paper_2511_15629_b300 import esdp as E
from paper_2511_15629_b300 import instances as I

pytestmark = pytest.mark.gpu
VTOL = 1e-5  # relative to max |V_1|, as in the parity tests


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    E.load_library()


def _inputs(inst):
    import torch
    cat = E.concat_inputs([inst])
    return {k: torch.from_numpy(v).cuda() for k, v in cat.items()}


@pytest.mark.parametrize("make", [I.config1, lambda: I.random_instance(90, 9, 333, 6, 17, 11, 2,
                                                                       neg_prob=0.3)])
def test_noalloc_matches_esdp_solve_twice(make):
    import torch
    inst = make()
    d = _inputs(inst)
    MNK = inst.n_modes * inst.N * inst.K
    ref = torch.empty(MNK, device="cuda")
    s = E.Solver([inst], device_ptrs=True)
    s.solve(d["price"], d["trans"], d["cost"], d["terminal"], ref)
    torch.cuda.synchronize()
    ref_pol = torch.empty(inst.T * MNK, dtype=torch.int32, device="cuda")
    for t in range(1, inst.T + 1):
        s.policy(0, t, ref_pol[(t - 1) * MNK:t * MNK])
    torch.cuda.synchronize()
    scale = float(ref.abs().max())
    for call in range(2):
        V1 = torch.full((MNK,), float("nan"), device="cuda")
        pol = torch.full((inst.T * MNK,), -7, dtype=torch.int32, device="cuda")
        E.solve_noalloc(inst, d["price"], d["trans"], d["cost"], d["terminal"], V1, pol)
        err = float((V1 - ref).abs().max()) / scale
        assert err <= VTOL, f"call {call}: rel error {err:.3e}"
        assert torch.equal(pol, ref_pol), f"call {call}: policies differ"
    s.close()


@pytest.mark.parametrize("K", [8, 16])
def test_noalloc_mma_path(monkeypatch, K):
    """The mma.sync EV contraction (pinned with ESDP_EV in both entry points,
    so both take the same arithmetic) gives the regular solve's values and
    policies."""
    import torch
    monkeypatch.setenv("ESDP_EV", "mma")
    inst = I.random_instance(92 + K, 6, 257, K, 15, 12, 2, neg_prob=0.3)
    d = _inputs(inst)
    MNK = inst.n_modes * inst.N * inst.K
    ref = torch.empty(MNK, device="cuda")
    s = E.Solver([inst], device_ptrs=True)
    assert s.launch_info()["ev"] == "mma.sync"
    s.solve(d["price"], d["trans"], d["cost"], d["terminal"], ref)
    ref_pol = torch.empty(inst.T * MNK, dtype=torch.int32, device="cuda")
    for t in range(1, inst.T + 1):
        s.policy(0, t, ref_pol[(t - 1) * MNK:t * MNK])
    torch.cuda.synchronize()
    V1 = torch.full((MNK,), float("nan"), device="cuda")
    pol = torch.full((inst.T * MNK,), -7, dtype=torch.int32, device="cuda")
    E.solve_noalloc(inst, d["price"], d["trans"], d["cost"], d["terminal"], V1, pol)
    err = float((V1 - ref).abs().max()) / float(ref.abs().max())
    assert err <= VTOL
    assert torch.equal(pol, ref_pol)
    s.close()


@pytest.mark.parametrize("K,modes", [(64, 1), (63, 2)])
def test_noalloc_fixed_stride_variant(monkeypatch, K, modes):
    """Assets with K = 63 or 64 run the sweep variant with a compile-time EV
    row stride inside the allocation-free entry point too; with the FP32
    SIMT contraction pinned in both entry points (the same arithmetic), it
    gives the regular solve's values and policies, on two calls in a row."""
    import torch
    monkeypatch.setenv("ESDP_EV", "simt")
    inst = I.random_instance(95 + K, 5, 410, K, 21, 17, modes, neg_prob=0.25,
                             cost="nonconvex")
    d = _inputs(inst)
    MNK = inst.n_modes * inst.N * inst.K
    ref = torch.empty(MNK, device="cuda")
    s = E.Solver([inst], device_ptrs=True)
    assert s.launch_info()["ev"] == "simt"
    s.solve(d["price"], d["trans"], d["cost"], d["terminal"], ref)
    ref_pol = torch.empty(inst.T * MNK, dtype=torch.int32, device="cuda")
    for t in range(1, inst.T + 1):
        s.policy(0, t, ref_pol[(t - 1) * MNK:t * MNK])
    torch.cuda.synchronize()
    s.close()
    scale = float(ref.abs().max())
    for call in range(2):
        V1 = torch.full((MNK,), float("nan"), device="cuda")
        pol = torch.full((inst.T * MNK,), -7, dtype=torch.int32, device="cuda")
        E.solve_noalloc(inst, d["price"], d["trans"], d["cost"], d["terminal"], V1, pol)
        err = float((V1 - ref).abs().max()) / scale
        assert err <= VTOL, f"call {call}: rel error {err:.3e}"
        assert torch.equal(pol, ref_pol), f"call {call}: policies differ"


def test_noalloc_allocates_no_device_memory():
    """After a first call (which loads the library's device code, and with
    it the fixed workspace, on this device), further calls change neither
    the device's free memory nor the caching allocator's reserved or
    allocated bytes: the entry point allocates nothing."""
    import torch
    inst = I.random_instance(93, 7, 300, 5, 12, 10, 2, neg_prob=0.3)
    d = _inputs(inst)
    MNK = inst.n_modes * inst.N * inst.K
    V1 = torch.empty(MNK, device="cuda")
    pol = torch.empty(inst.T * MNK, dtype=torch.int32, device="cuda")
    E.solve_noalloc(inst, d["price"], d["trans"], d["cost"], d["terminal"], V1, pol)
    first = V1.clone()
    torch.cuda.synchronize()
    before = (torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved(),
              torch.cuda.memory_allocated())
    for _ in range(3):
        E.solve_noalloc(inst, d["price"], d["trans"], d["cost"], d["terminal"], V1, pol)
    torch.cuda.synchronize()
    after = (torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved(),
             torch.cuda.memory_allocated())
    assert after == before, f"device memory (free, reserved, allocated) {before} -> {after}"
    assert torch.equal(V1, first)


def test_noalloc_bounded_wait_times_out(monkeypatch):
    """The allocation-free entry point's device waits are bounded like the
    context's: with every wait made to wait for a flag value nothing
    publishes (the ESDP_INJECT_STALL test hook) and a 300 ms limit, the call
    returns ESDP_ETIMEOUT, and the next call on the same workspace is
    correct again (the flags and the status word are cleared per call)."""
    import torch
    inst = I.random_instance(94, 5, 200, 4, 9, 9, 1, neg_prob=0.2)
    d = _inputs(inst)
    MNK = inst.n_modes * inst.N * inst.K
    ref = torch.empty(MNK, device="cuda")
    s = E.Solver([inst], device_ptrs=True)
    s.solve(d["price"], d["trans"], d["cost"], d["terminal"], ref)
    torch.cuda.synchronize()
    s.close()
    V1 = torch.empty(MNK, device="cuda")
    monkeypatch.setenv("ESDP_TIMEOUT_MS", "300")
    monkeypatch.setenv("ESDP_INJECT_STALL", "1")
    with pytest.raises(E.EsdpError) as ei:
        E.solve_noalloc(inst, d["price"], d["trans"], d["cost"], d["terminal"], V1)
    assert ei.value.code == E.ESDP_ETIMEOUT
    monkeypatch.delenv("ESDP_INJECT_STALL")
    E.solve_noalloc(inst, d["price"], d["trans"], d["cost"], d["terminal"], V1)
    err = float((V1 - ref).abs().max()) / float(ref.abs().max())
    assert err <= VTOL


def test_noalloc_rejects_assets_beyond_the_workspace():
    import torch
    inst = I.random_instance(91, 2, 40000, 64, 3, 3, 1)
    d = _inputs(inst)
    V1 = torch.empty(inst.N * inst.K, device="cuda")
    with pytest.raises(E.EsdpError) as ei:
        E.solve_noalloc(inst, d["price"], d["trans"], d["cost"], d["terminal"], V1)
    assert ei.value.code == E.ESDP_EINVAL
    assert "bytes of workspace" in str(ei.value)
