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


def test_noalloc_rejects_assets_beyond_the_workspace():
    import torch
    inst = I.random_instance(91, 2, 40000, 64, 3, 3, 1)
    d = _inputs(inst)
    V1 = torch.empty(inst.N * inst.K, device="cuda")
    with pytest.raises(E.EsdpError) as ei:
        E.solve_noalloc(inst, d["price"], d["trans"], d["cost"], d["terminal"], V1)
    assert ei.value.code == E.ESDP_EINVAL
    assert "bytes of workspace" in str(ei.value)
