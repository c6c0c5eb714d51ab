"""GPU (CUDA library, through the C ABI) against the FP64 oracle.

Bars (stated for the method):
  * values: max |V_gpu - V_oracle| <= 1e-5 * max |V_1 oracle|;
  * policies: identical wherever the oracle's top-two action gap is at least
    1e-6 * max |V_1| (near-ties may resolve either way in float32);
  * bid-curve vertices: bit-exact against the oracle envelope run on the
    GPU's own float32 EV; slopes within float32 rounding;
  * gradients: max |g_gpu - g_oracle| <= 1e-4 * max |g_oracle| per tensor.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_15629_b300 import build as B
from paper_2511_15629_b300 import esdp as E
from paper_2511_15629_b300 import instances as I

pytestmark = pytest.mark.gpu
NTHREADS = max(1, len(os.sched_getaffinity(0)))
VTOL = 1e-5
GAPTOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    E.load_library()


def _scale(V1):
    return max(float(np.abs(V1).max()), 1e-12)


def assert_values(gpu, ref, scale, what="V"):
    err = float(np.abs(gpu.astype(np.float64) - ref).max()) / scale
    assert err <= VTOL, f"{what}: max rel error {err:.3e} > {VTOL}"
    return err


def assert_policy(gpu, ref, gap, scale, what="policy", inst=None, EV=None, t0=1):
    """Policies [n_t, M, N, K] of stages t0, t0+1, ...: identical wherever
    the oracle's top-two gap is at least GAPTOL * scale.  Inside that band
    several actions are maximisers to float32 accuracy; with the instance and
    the FP64 EV of those stages (`EV` [n_t, M, N, K]) every GPU decision that
    differs from the oracle's is evaluated by the oracle (payoff + EV at the
    shifted SoC) and must lie within GAPTOL * scale of the best value.
    Returns the number of differing near-tie decisions."""
    gpu = np.asarray(gpu).reshape(np.shape(ref))
    decided = gap >= GAPTOL * scale
    differ = gpu.astype(np.int64) != ref.astype(np.int64)
    bad = differ & decided
    assert not bad.any(), f"{what}: {int(bad.sum())} mismatches outside near-ties"
    near = differ & ~decided
    if inst is not None and EV is not None and near.any():
        ti, m, si, k = np.nonzero(near)
        for tt in np.unique(ti):
            sel = ti == tt
            t = t0 + int(tt)
            a_gpu = gpu[tt, m[sel], si[sel], k[sel]].astype(np.int64)
            a_ref = ref[tt, m[sel], si[sel], k[sel]].astype(np.int64)
            q_gpu = O.action_value(inst, t, EV[tt], m[sel], si[sel], k[sel], a_gpu)
            q_best = O.action_value(inst, t, EV[tt], m[sel], si[sel], k[sel], a_ref)
            short = float((q_best - q_gpu).max())
            assert short <= GAPTOL * scale, \
                f"{what}: stage {t} near-tie decision {short:.3e} below the best " \
                f"(> {GAPTOL} * {scale:.3e})"
    return int(near.sum())


def solve_gpu(inst, keep_ev=False, tune=False):
    """Solve on the GPU; tune=True first times the launch shapes as bench.py
    does, so that the benchmark's launch configuration is the one checked."""
    s = E.Solver([inst], keep_ev=keep_ev)
    if tune:
        s.autotune()
    V1 = s.solve_instances()[0]
    return s, V1


def gpu_policies(s, inst):
    return np.stack([s.policy(0, t) for t in range(1, inst.T + 1)])


def full_check(inst, keep_ev=False, check_policy=True, tune=False):
    s, V1 = solve_gpu(inst, keep_ev=keep_ev, tune=tune)
    want_pol = check_policy and inst.policy_bytes and not inst.ckpt_every
    r = O.solve(inst, keep_EV=keep_ev or want_pol, nthreads=NTHREADS)
    scale = _scale(r["V1"])
    assert_values(V1, r["V1"], scale)
    if want_pol:
        assert_policy(gpu_policies(s, inst), r["policy"], r["gap"], scale, inst=inst, EV=r["EV"])
    if keep_ev:
        ev = np.stack([s.expected_value(0, t) for t in range(1, inst.T + 1)])
        assert_values(ev, r["EV"], scale, "EV")
    return s, r


# ----------------------------------------------------------------- sweep

def test_config1_parity():
    full_check(I.config1(), keep_ev=True)


RANDOM_CASES = [
    # T, N, K, D_dis, D_chg, modes, seed, cost
    (5, 2, 1, 1, 0, 1, 1, "linear"),        # smallest grid
    (7, 37, 3, 5, 2, 1, 2, "nonconvex"),    # ragged, asymmetric band
    (6, 300, 33, 20, 17, 1, 3, "linear"),   # K not a multiple of the warp
    (4, 129, 8, 64, 64, 2, 4, "nonconvex"), # band wider than a tile, two modes
    (9, 50, 1, 49, 49, 1, 5, "linear"),     # band spans the whole grid
    (3, 1000, 2, 0, 0, 1, 6, "zero"),       # idle only
    (5, 64, 7, 0, 9, 2, 7, "linear"),       # charge-only band with modes
    (5, 64, 7, 9, 0, 2, 8, "linear"),       # discharge-only band with modes
    (12, 777, 16, 33, 31, 2, 9, "nonconvex"),
    (2, 5001, 5, 100, 100, 1, 10, "linear"),
    (3, 200, 128, 10, 10, 2, 11, "nonconvex"),  # largest K: tensor-core EV, two modes
    (3, 150, 127, 7, 9, 1, 12, "linear"),       # largest odd K (SIMT EV)
    (3, 2000, 4, 600, 700, 1, 13, "linear"),    # A = 1301: a very wide band
]


@pytest.mark.parametrize("case", RANDOM_CASES, ids=[f"T{c[0]}N{c[1]}K{c[2]}D{c[3]}-{c[4]}M{c[5]}"
                                                     for c in RANDOM_CASES])
def test_random_shapes_parity(case):
    T, N, K, Dd, Dc, M, seed, cost = case
    inst = I.random_instance(seed, T, N, K, Dd, Dc, M, neg_prob=0.25, cost=cost,
                             switch_cost=4.0)
    full_check(inst, keep_ev=True)


def test_ties_resolve_to_smallest_action():
    inst = I.random_instance(11, 4, 40, 3, 6, 6, 1, cost="zero", terminal="zero")
    inst.price[:] = 0
    s, V1 = solve_gpu(inst)
    pol = gpu_policies(s, inst)
    assert np.all(V1 == 0)
    for si in range(inst.N):
        assert np.all(pol[:, 0, si, :] == max(0, inst.D_dis - si))


def test_integer_prices_exact_ties():
    """Integer prices and a linear terminal give many exact float ties; the
    GPU must still return the smallest maximiser of its own float values."""
    inst = I.random_instance(12, 6, 90, 4, 7, 7, 2, integer_prices=True, cost="zero",
                             terminal="linear", eta=(1.0, 1.0), s_max=90 * 0.25)
    s, r = full_check(inst, keep_ev=True)


def test_config2_parity_with_modes():
    full_check(I.config2(), keep_ev=True, tune=True)


def test_config5_values_int16_checkpointed():
    inst = I.config5()
    s, V1 = solve_gpu(inst, tune=True)
    r = O.solve(inst, nthreads=NTHREADS, keep_policy=False)
    assert_values(V1, r["V1"], _scale(r["V1"]))
    with pytest.raises(E.EsdpError) as ei:
        s.policy(0, 1)              # checkpointed: no full policy kept
    assert ei.value.code == E.ESDP_ESTATE


def test_int16_full_policy_matches_int32():
    a = I.random_instance(13, 8, 200, 6, 12, 12, 2)
    b = I.random_instance(13, 8, 200, 6, 12, 12, 2)
    b.policy_bytes = 2
    sa, Va = solve_gpu(a)
    sb, Vb = solve_gpu(b)
    np.testing.assert_array_equal(Va, Vb)
    np.testing.assert_array_equal(gpu_policies(sa, a), gpu_policies(sb, b).astype(np.int32))


def _c3_last(nstages):
    inst = I.config3()
    return I.Instance("config3_tail", nstages, inst.N, inst.K, inst.A, inst.D_dis, inst.D_chg, 1,
                      inst.s_max, inst.tau, inst.eta_c, inst.eta_d, 0.0,
                      inst.price[-nstages:].copy(), inst.trans[-nstages:].copy(), inst.cost,
                      inst.terminal, s0=inst.s0)


def test_config3_tail_full_parity():
    """Full-width C3 stages (N=5001, K=64, A=201) over the last 12 stages."""
    full_check(_c3_last(12), keep_ev=True)


def test_fixed_row_stride_variant_equals_runtime_stride(monkeypatch):
    """K = 64 assets run the sweep variant whose EV tile row stride is a
    compile-time constant; the variant that reads it at run time (pinned
    with ESDP_NO_KH) gives the same bits."""
    inst = _c3_last(6)
    a = solve_gpu(inst)[1]
    monkeypatch.setenv("ESDP_NO_KH", "1")
    b = solve_gpu(inst)[1]
    np.testing.assert_array_equal(a, b)
    odd = I.random_instance(97, 4, 400, 63, 30, 25, 2, neg_prob=0.2, cost="nonconvex")
    c = solve_gpu(odd)[1]
    monkeypatch.delenv("ESDP_NO_KH")
    d = solve_gpu(odd)[1]
    np.testing.assert_array_equal(c, d)
    r = O.solve(odd, nthreads=NTHREADS, keep_policy=False)
    assert_values(d, r["V1"], _scale(r["V1"]))


def test_config3_full_horizon_sampled_stages():
    """The C3 sweep in its benchmark launch shape (all 2016 stages, keep EV).
    Each sampled stage is checked against the oracle's Bellman step taken
    from the GPU's own EV_t; V_1 against the full FP64 oracle."""
    inst = I.config3()
    s = E.Solver([inst], keep_ev=True)
    s.autotune()
    V1 = s.solve_instances()[0]
    for t in (inst.T, 1500, 700, 2):
        ev_t = s.expected_value(0, t).astype(np.float64)
        ev_prev = s.expected_value(0, t - 1).astype(np.float64)
        r1 = _bellman_from_ev(inst, t, ev_t)
        Vt, pol, gap = r1
        scale = float(np.abs(Vt).max())
        P = inst.trans[t - 2].astype(np.float64)
        np.testing.assert_array_less(np.abs(Vt @ P.T - ev_prev).max() / scale, VTOL)
        pg = s.policy(0, t)[0]
        assert_policy(pg[None, None], pol[None, None], gap[None, None], scale, f"policy t={t}",
                      inst=inst, EV=ev_t[None], t0=t)
    r = O.solve(inst, nthreads=NTHREADS, keep_policy=False)
    assert_values(V1, r["V1"], _scale(r["V1"]))


def _bellman_from_ev(inst, t, ev):
    """Oracle Bellman step of stage t (eq. 5) from a given EV_t [1,N,K]."""
    tmp = I.Instance("one", 1, inst.N, inst.K, inst.A, inst.D_dis, inst.D_chg, 1, inst.s_max,
                     inst.tau, inst.eta_c, inst.eta_d, 0.0, inst.price[t - 1:t].copy(),
                     np.eye(inst.K, dtype=np.float32)[None], inst.cost,
                     np.zeros((1, inst.N, inst.K), np.float32))
    # identity transition: EV_1 = V_2 = terminal, so pass ev as the terminal
    r = O.solve(tmp, terminal=ev, nthreads=NTHREADS)
    return r["V1"][0], r["policy"][0, 0], r["gap"][0, 0]


# ------------------------------------------------------------ bid curves

@pytest.mark.parametrize("which", ["config2", "random"])
def test_bid_curves_bit_exact(which):
    inst = I.config2() if which == "config2" else I.random_instance(21, 9, 400, 6, 25, 30, 1,
                                                                     neg_prob=0.4,
                                                                     cost="nonconvex")
    s, V1 = solve_gpu(inst, keep_ev=True)
    n_bp, idx, slope = s.bid_curves(0, 1, inst.T + 1)
    ev = np.stack([s.expected_value(0, t) for t in range(1, inst.T + 1)])
    ref_n, ref_idx, ref_slope = O.bid_curves(inst, ev)
    np.testing.assert_array_equal(n_bp, ref_n)
    for t in range(inst.T):
        for m in range(inst.n_modes):
            for k in range(inst.K):
                n = n_bp[t, m, k]
                np.testing.assert_array_equal(idx[t, m, k, :n], ref_idx[t, m, k, :n])
                np.testing.assert_allclose(slope[t, m, k, :n - 1], ref_slope[t, m, k, :n - 1],
                                           rtol=1e-6, atol=1e-6)
                # monotone bids: strictly decreasing in double, and no float32
                # rounding can reverse the order
                assert np.all(np.diff(ref_slope[t, m, k, :n - 1]) < 0)
                assert np.all(np.diff(slope[t, m, k, :n - 1]) <= 0)


def test_bid_curves_against_fp64_envelope():
    """Against the envelope of the oracle's FP64 EV: vertices may differ only
    where a vertex is nearly collinear with its neighbours."""
    inst = I.config2()
    s, V1 = solve_gpu(inst, keep_ev=True)
    n_bp, idx, slope = s.bid_curves(0, 1, inst.T + 1)
    r = O.solve(inst, keep_EV=True, nthreads=NTHREADS, keep_policy=False)
    ref_n, ref_idx, _ = O.bid_curves(inst, r["EV"])
    same = 0
    for t in range(inst.T):
        for m in range(inst.n_modes):
            for k in range(inst.K):
                a = idx[t, m, k, :n_bp[t, m, k]]
                b = ref_idx[t, m, k, :ref_n[t, m, k]]
                if len(a) == len(b) and np.array_equal(a, b):
                    same += 1
                    continue
                # envelopes agree to float32 accuracy even where vertices differ
                y = r["EV"][t, m, :, k]
                ea = np.interp(np.arange(inst.N), a, y[a])
                eb = np.interp(np.arange(inst.N), b, y[b])
                assert np.abs(ea - eb).max() <= 1e-6 * np.abs(y).max() + 1e-9
    total = inst.T * inst.n_modes * inst.K
    print(f"identical vertex sets vs the FP64-EV envelope: {same}/{total}")
    assert same >= 0.5 * total


# ------------------------------------------------------------- gradients

def _gpu_full_policy(inst):
    """The GPU's own stored argmax decisions for every stage (same values as a
    checkpointed solve of the instance: the sweep is deterministic)."""
    import copy
    full = copy.copy(inst)
    full.ckpt_every = 0
    s, _ = solve_gpu(full)
    return gpu_policies(s, full).astype(np.int32)


def _grad_check(inst, tie_free, tune=False):
    s, V1 = solve_gpu(inst, tune=tune)
    J, dp, dt, de, dco, dsw, dterm, dmu = s.grad(0, inst.mu0, extra=True)
    r = O.solve(inst, keep_V=True, keep_EV=True, nthreads=NTHREADS)
    scale = _scale(r["V1"])
    pol = _gpu_full_policy(inst)
    n_near_tie = assert_policy(pol, r["policy"], r["gap"], scale, inst=inst, EV=r["EV"])
    # the bar: FP64 occupancy pass under the same decisions as the GPU
    occ = O.occupancy(inst, pol, r["V"])
    assert J[0] == pytest.approx(occ["J"], rel=VTOL)
    checks = (("d_price", dp, "d_price"), ("d_trans", dt, "d_trans"),
              ("d_eta_c", de[:1], "d_eta_c"), ("d_eta_d", de[1:], "d_eta_d"),
              ("d_cost", dco, "d_cost"), ("d_terminal", dterm, "d_terminal"),
              ("d_mu0", dmu, "d_mu0"))
    if inst.n_modes == 2:
        checks += (("d_switch", dsw, "d_switch"),)
    else:
        assert dsw[0] == 0.0
    for name, g, key in checks:
        ref = np.atleast_1d(occ[key])
        err = np.abs(g.astype(np.float64).reshape(ref.shape) - ref).max() / max(np.abs(ref).max(), 1e-12)
        assert err <= 1e-4, f"{name}: rel error {err:.3e}"
    if tie_free:
        # no near-ties: the oracle's own decisions give the same gradient
        assert n_near_tie == 0
        occ2 = O.occupancy(inst, r["policy"], r["V"])
        for name, g, key in checks:
            ref = np.atleast_1d(occ2[key])
            err = np.abs(g.astype(np.float64).reshape(ref.shape) - ref).max() / max(np.abs(ref).max(), 1e-12)
            assert err <= 1e-4, f"{name} (oracle decisions): rel error {err:.3e}"
    return n_near_tie


def test_gradient_small_tie_free():
    inst = I.random_instance(53, 6, 25, 3, 3, 3, 1, neg_prob=0.2, cost="linear")
    inst.s0 = 12
    _grad_check(inst, tie_free=True)


def test_gradient_modes_checkpointed():
    inst = I.random_instance(54, 40, 120, 5, 9, 9, 2, neg_prob=0.2, switch_cost=3.0)
    inst.s0 = 60
    inst.ckpt_every = 7
    inst.policy_bytes = 2
    _grad_check(inst, tie_free=False)


def test_gradient_repeat_calls_agree():
    """Two gradient calls on the same solve give the same bits: the
    occupancy scatter adds in fixed point (associative integer atomics) and
    every other sum runs in a fixed order."""
    inst = I.random_instance(55, 30, 150, 6, 10, 12, 2, neg_prob=0.2, switch_cost=3.0)
    inst.s0 = 70
    inst.ckpt_every = 8
    s, _ = solve_gpu(inst)
    mu0 = np.full(inst.K, 1.0 / inst.K, np.float32)
    a = s.grad(0, mu0, extra=True)
    b = s.grad(0, mu0, extra=True)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))


def test_gradient_segment_groups_agree(monkeypatch):
    """The checkpoint segments are re-swept B at a time as the assets of one
    launch (ESDP_GRAD_SEGMENTS = B; 5 segments: groups 5, 3 + 2, 2 + 2 + 1
    and 1 at a time).  Every grouping gives the same bits: a segment's
    recomputation does not depend on the segments launched beside it (K = 10
    keeps every tile on the FP32 SIMT contraction)."""
    inst = I.random_instance(57, 37, 260, 10, 12, 14, 2, neg_prob=0.2, switch_cost=3.0)
    inst.s0 = 120
    inst.ckpt_every = 8
    inst.policy_bytes = 2
    s, _ = solve_gpu(inst)
    mu0 = np.full(inst.K, 1.0 / inst.K, np.float32)
    ref = None
    for b in ("5", "3", "2", "1"):
        monkeypatch.setenv("ESDP_GRAD_SEGMENTS", b)
        out = s.grad(0, mu0, extra=True)
        if ref is None:
            ref = out
            continue
        for x, y in zip(ref, out):
            np.testing.assert_array_equal(np.asarray(x), np.asarray(y))


def test_gradient_segment_groups_on_tensor_path(monkeypatch):
    """The grouped segment re-sweeps with the EV contraction pinned to
    tcgen05 (K = 16): the gradient matches the FP64 occupancy pass under the
    GPU's decisions, and re-sweeping the four segments one at a time gives
    the same bits as all four in one launch."""
    monkeypatch.setenv("ESDP_EV", "tc")
    inst = I.random_instance(58, 22, 180, 16, 10, 12, 1, neg_prob=0.2)
    inst.s0 = 90
    inst.ckpt_every = 6
    inst.policy_bytes = 2
    _grad_check(inst, tie_free=False)
    s, _ = solve_gpu(inst)
    assert s.launch_info()["ev"] == "tcgen05"
    mu0 = np.full(inst.K, 1.0 / inst.K, np.float32)
    ref = s.grad(0, mu0, extra=True)
    monkeypatch.setenv("ESDP_GRAD_SEGMENTS", "1")
    one = s.grad(0, mu0, extra=True)
    for x, y in zip(ref, one):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))


def test_batch_variant_odd_states_values_and_policies():
    """Assets with K not a multiple of 4 (odd K, one and two modes) run the
    batch variant of the sweep kernel: its EV-tile copy, its one-part argmax
    recovery and its flat output stores.  Values and stored decisions of
    every stage match the FP64 oracle."""
    assets = [I.random_instance(90 + j, 9, n, k, d1, d2, m, neg_prob=0.2)
              for j, (n, k, d1, d2, m) in enumerate([(230, 5, 14, 11, 1), (161, 7, 9, 9, 2),
                                                     (97, 9, 20, 6, 1), (301, 3, 4, 30, 2),
                                                     (64, 11, 8, 8, 1)])]
    s = E.Solver(assets)
    V1s = s.solve_instances()
    for j, (inst, V1) in enumerate(zip(assets, V1s)):
        r = O.solve(inst, keep_EV=True, nthreads=NTHREADS)
        scale = _scale(r["V1"])
        assert_values(V1, r["V1"], scale, inst.name)
        pol = np.stack([s.policy(j, t) for t in range(1, inst.T + 1)])
        assert_policy(pol, r["policy"], r["gap"], scale, what=f"{inst.name} policy",
                      inst=inst, EV=r["EV"])


def test_gradient_rejects_occupancy_beyond_fixed_point_range():
    """An initial distribution with entries above 2^20 cannot be added in the
    scatter's fixed point: the call reports ESDP_ENUMERIC instead of
    wrapping around."""
    inst = I.random_instance(56, 6, 80, 4, 5, 5, 1)
    inst.s0 = 40
    s, _ = solve_gpu(inst)
    with pytest.raises(E.EsdpError) as ei:
        s.grad(0, np.full(inst.K, 4.0e6, np.float32))
    assert ei.value.code == E.ESDP_ENUMERIC
    J = s.grad(0, inst.mu0)[0]  # the context stays usable
    assert np.isfinite(J).all()


def test_gradient_config5():
    n = _grad_check(I.config5(), tie_free=False, tune=True)
    print(f"config5: {n} near-tie decisions differ from the FP64 oracle's")


# --------------------------------------------------------------- batching

def test_batched_equals_solo_and_oracle():
    assets = [I.random_instance(60 + j, 10, n, k, d1, d2, m, neg_prob=0.2)
              for j, (n, k, d1, d2, m) in enumerate([(300, 8, 20, 20, 1), (77, 3, 5, 9, 2),
                                                     (1001, 12, 40, 40, 1), (2, 1, 1, 1, 1),
                                                     (450, 40, 60, 50, 1), (130, 5, 3, 3, 2)])]
    s = E.Solver(assets)
    V1s = s.solve_instances()
    for inst, V1 in zip(assets, V1s):
        _, solo = solve_gpu(inst)
        np.testing.assert_array_equal(V1, solo)
        r = O.solve(inst, nthreads=NTHREADS, keep_policy=False)
        assert_values(V1, r["V1"], _scale(r["V1"]))


def test_config4_subset_truncated_horizon():
    """16 portfolio assets with their full N, K, A on a 24-stage horizon."""
    assets = []
    for j in range(16):
        a = I.config4_asset(j)
        a.T = 24
        a.price = np.ascontiguousarray(a.price[:24])
        a.trans = np.ascontiguousarray(a.trans[:24])
        assets.append(a)
    s = E.Solver(assets)
    for inst, V1 in zip(assets, s.solve_instances()):
        r = O.solve(inst, nthreads=NTHREADS, keep_policy=False)
        assert_values(V1, r["V1"], _scale(r["V1"]), inst.name)


def test_config4_benchmarked_launch_equals_solo_and_oracle():
    """The portfolio launch exactly as the benchmark times it: all 256
    assets at the full T = 288, tile shapes picked by autotune(), one
    graph-captured persistent launch on device pointers.  Every asset's V_1
    equals its own single-asset solve bit for bit (K <= 40: the EV
    contraction is FP32 SIMT with the same summation order in both plans),
    and a seeded subset of 12 assets matches the FP64 oracle over the full
    horizon."""
    import torch
    assets = I.config4(256)
    cat = E.concat_inputs(assets)
    d = {k: torch.from_numpy(v).cuda() for k, v in cat.items()}
    sizes = [a.n_modes * a.N * a.K for a in assets]
    V1 = torch.empty(sum(sizes), device="cuda")
    s = E.Solver(assets, device_ptrs=True)
    s.autotune()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s.solve(d["price"], d["trans"], d["cost"], d["terminal"], V1, stream=st)
    st.synchronize()
    g = torch.cuda.CUDAGraph()
    V1.fill_(float("nan"))
    with torch.cuda.graph(g, stream=st):
        s.solve(d["price"], d["trans"], d["cost"], d["terminal"], V1,
                stream=torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    assert s.status(stream=st) == 0
    got = np.split(V1.cpu().numpy(), np.cumsum(sizes)[:-1])
    info = s.launch_info()
    s.close()
    for j, inst in enumerate(assets):
        _, solo = solve_gpu(inst)
        np.testing.assert_array_equal(got[j], solo.reshape(-1), err_msg=f"asset {j} ({info})")
    for j in np.random.default_rng(404).choice(256, size=12, replace=False):
        inst = assets[j]
        r = O.solve(inst, nthreads=NTHREADS, keep_policy=False)
        assert_values(got[j].reshape(r["V1"].shape), r["V1"], _scale(r["V1"]), inst.name)


@pytest.mark.parametrize("world", [2, 4])
def test_portfolio_shards_equal_full_batch(world):
    """Multi-GPU asset sharding, on one GPU: each rank's share of the
    portfolio (dist.shard_by_cost, longest processing time first) solved in
    a context of its own reproduces the full batch's V_1 of those assets bit
    for bit, so the shards can run on separate GPUs with no collective."""
    from paper_2511_15629_b300 import dist as D
    assets = []
    for j in range(24):
        a = I.config4_asset(j)
        a.T = 48
        a.price = np.ascontiguousarray(a.price[:48])
        a.trans = np.ascontiguousarray(a.trans[:48])
        assets.append(a)
    full = E.Solver(assets).solve_instances()
    shards = D.shard_by_cost([a.evals for a in assets], world)
    assert sorted(i for sh in shards for i in sh) == list(range(len(assets)))
    for sh in shards:
        assert sh, "every rank gets assets"
        part = E.Solver([assets[i] for i in sh]).solve_instances()
        for i, V in zip(sh, part):
            np.testing.assert_array_equal(V, full[i], err_msg=f"asset {i}, world {world}")


# ---------------------------------------------------- device mode / errors

def test_device_pointers_and_graph_capture():
    import torch
    inst = I.random_instance(70, 20, 500, 10, 30, 30, 2)
    cat = E.concat_inputs([inst])
    dev = {k: torch.from_numpy(v).cuda() for k, v in cat.items()}
    V1 = torch.empty(inst.n_modes * inst.N * inst.K, device="cuda")
    s = E.Solver([inst], device_ptrs=True)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s.solve(dev["price"], dev["trans"], dev["cost"], dev["terminal"], V1, stream=st)
    st.synchronize()
    assert s.status(stream=st) == 0
    _, ref = solve_gpu(inst)
    np.testing.assert_array_equal(V1.cpu().numpy().reshape(ref.shape), ref)
    # capture the solve in a CUDA graph and replay it on new prices
    g = torch.cuda.CUDAGraph()
    V2 = torch.zeros_like(V1)
    with torch.cuda.graph(g, stream=st):
        s.solve(dev["price"], dev["trans"], dev["cost"], dev["terminal"], V2,
                stream=torch.cuda.current_stream())
    dev["price"].mul_(1.5)
    g.replay()
    torch.cuda.synchronize()
    inst2 = I.random_instance(70, 20, 500, 10, 30, 30, 2)
    inst2.price = (inst2.price * np.float32(1.5)).astype(np.float32)
    _, ref2 = solve_gpu(inst2)
    np.testing.assert_array_equal(V2.cpu().numpy().reshape(ref2.shape), ref2)


def test_bad_inputs_rejected():
    inst = I.random_instance(71, 4, 50, 3, 4, 4, 1)
    s = E.Solver([inst])
    cat = E.concat_inputs([inst])
    with pytest.raises(E.EsdpError) as ei:
        s.policy(0, 1)
    assert ei.value.code == E.ESDP_ESTATE
    bad = dict(cat)
    bad["price"] = cat["price"].copy()
    bad["price"][3] = np.nan
    with pytest.raises(E.EsdpError) as ei:
        s.solve(bad["price"], bad["trans"], bad["cost"], bad["terminal"])
    assert ei.value.code == E.ESDP_EINVAL
    bad = dict(cat)
    bad["trans"] = cat["trans"].copy()
    bad["trans"][5] = -0.1
    with pytest.raises(E.EsdpError) as ei:
        s.solve(bad["price"], bad["trans"], bad["cost"], bad["terminal"])
    assert ei.value.code == E.ESDP_EINVAL
    with pytest.raises(E.EsdpError) as ei:
        s.bid_curves(0, 1, 2)
    assert ei.value.code in (E.ESDP_ESTATE,)
    s.solve(cat["price"], cat["trans"], cat["cost"], cat["terminal"])  # still usable
    with pytest.raises(E.EsdpError) as ei:
        s.policy(0, inst.T + 1)
    assert ei.value.code == E.ESDP_EINVAL


def test_bounded_wait_times_out_and_context_recovers(monkeypatch):
    """Every neighbour wait is made to wait for a flag value nothing
    publishes; the bounded spin must give up, report ESDP_ETIMEOUT through
    the status word, and leave the context usable."""
    monkeypatch.setenv("ESDP_TIMEOUT_MS", "300")
    inst = I.random_instance(72, 6, 400, 4, 10, 10, 1)
    s = E.Solver([inst])
    cat = E.concat_inputs([inst])
    monkeypatch.setenv("ESDP_INJECT_STALL", "1")
    with pytest.raises(E.EsdpError) as ei:
        s.solve(cat["price"], cat["trans"], cat["cost"], cat["terminal"])
    assert ei.value.code == E.ESDP_ETIMEOUT
    monkeypatch.delenv("ESDP_INJECT_STALL")
    V1 = np.empty(inst.N * inst.K, np.float32)
    s.solve(cat["price"], cat["trans"], cat["cost"], cat["terminal"], V1)
    r = O.solve(inst, keep_policy=False)
    assert_values(V1.reshape(1, inst.N, inst.K), r["V1"], _scale(r["V1"]))


def test_autotune_keeps_results():
    inst = I.random_instance(73, 12, 900, 16, 40, 40, 1)
    s, V1 = solve_gpu(inst)
    s.autotune()
    V1b = s.solve_instances()[0]
    np.testing.assert_array_equal(V1, V1b)
    info = s.launch_info()
    assert info["grid"] >= 1 and info["rows_per_thread"] in (4, 6, 8, 9, 10, 12)


# ------------------------------------------------- bid-curve exact predicate

def _hull_gpu_vs_oracle(inst):
    s, V1 = solve_gpu(inst, keep_ev=True)
    n_bp, idx, slope = s.bid_curves(0, 1, inst.T + 1)
    ev = np.stack([s.expected_value(0, t) for t in range(1, inst.T + 1)])
    ref_n, ref_idx, _ = O.bid_curves(inst, ev)
    np.testing.assert_array_equal(n_bp, ref_n)
    for t in range(inst.T):
        for m in range(inst.n_modes):
            for k in range(inst.K):
                n = n_bp[t, m, k]
                np.testing.assert_array_equal(idx[t, m, k, :n], ref_idx[t, m, k, :n])
    return ev


def test_bid_curves_exact_collinear():
    """Zero prices and costs with a linear terminal value: EV is exactly linear
    in SoC in float32 (small integers), every middle point is collinear and
    the orientation test must take its exact route.  (The level offsets and
    the float32 row sums perturb a few values by an ulp.)"""
    inst = I.random_instance(80, 3, 300, 4, 5, 5, 1, cost="zero", terminal="linear",
                             s_max=299.0, eta=(1.0, 1.0))
    inst.price[:] = 0
    inst.terminal[:] = (np.arange(inst.N, dtype=np.float32) * np.float32(0.5))[None, :, None]
    ev = _hull_gpu_vs_oracle(inst).astype(np.float64)
    # most consecutive triples are exactly collinear (differences are exact
    # in double for these float32 values), so the exact route decided them
    d = np.diff(ev, axis=2)
    assert np.mean(d[:, :, 1:, :] == d[:, :, :-1, :]) > 0.5


def test_bid_curves_wide_dynamic_range():
    """Values spanning many binary orders of magnitude (tiny next to large)
    exercise the double route of the exact orientation test."""
    inst = I.random_instance(81, 2, 200, 3, 3, 3, 1, cost="zero", terminal="random")
    rng = np.random.default_rng(5)
    term = rng.uniform(-1, 1, size=inst.terminal.shape) * 10.0 ** rng.integers(-12, 6, size=inst.terminal.shape)
    inst.terminal[:] = term.astype(np.float32)
    inst.price[:] = np.float32(1e-6)
    _hull_gpu_vs_oracle(inst)


@pytest.mark.parametrize("N", [2, 5, 33, 97, 1025, 13001])
@pytest.mark.parametrize("shape", ["concave", "convex", "wave"])
def test_bid_curves_envelope_shapes(N, shape):
    """Envelopes whose every point is a vertex (concave), with only the end
    points as vertices (convex) or with alternating runs (wave), on grids
    narrower than a warp and wider than 32 points per lane: the bridges
    between partial hulls cross many empty and trimmed parts.  The longest
    grid does not fit the staged kernel's shared memory and runs the in-place
    variant."""
    D = min(2, N - 1)
    inst = I.random_instance(90 + N, 2, N, 3, D, D, 1, cost="zero", terminal="random")
    x = np.linspace(-1.0, 1.0, N)
    f = {"concave": -x * x, "convex": x * x, "wave": np.sin(7.0 * x) + 0.3 * x}[shape]
    inst.terminal[:] = (100.0 * f).astype(np.float32)[None, :, None]
    inst.price[:] = np.float32(0.0)
    _hull_gpu_vs_oracle(inst)


def test_autotune_shape_pin(monkeypatch):
    """ESDP_SHAPE pins the launch shape (no timing); a malformed value is
    rejected; results do not depend on the shape."""
    inst = I.random_instance(77, 9, 333, 7, 13, 17, 1)
    ref = solve_gpu(inst)[1]
    monkeypatch.setenv("ESDP_SHAPE", "6,384")
    s = E.Solver([inst])
    s.autotune()
    info = s.launch_info()
    assert info["rows_per_thread"] == 6 and info["block"] == 384
    V1 = s.solve_instances()[0]
    np.testing.assert_allclose(V1, ref, rtol=0, atol=1e-5 * np.abs(ref).max())
    monkeypatch.setenv("ESDP_SHAPE", "six")
    with pytest.raises(E.EsdpError) as ei:
        E.Solver([inst]).autotune()
    assert ei.value.code == E.ESDP_EINVAL


@pytest.mark.parametrize("R,block,K", [(4, 256, 20), (6, 512, 20), (8, 256, 16), (9, 512, 20),
                                       (9, 256, 16), (10, 384, 20), (12, 256, 12)])
def test_every_rows_per_thread_variant(monkeypatch, R, block, K):
    """Each compiled rows-per-thread variant of the sweep (pinned through
    ESDP_SHAPE) matches the oracle's values and policies; K = 16 takes the
    tcgen05 EV path (pinned through ESDP_EV), the others SIMT."""
    inst = I.random_instance(90 + R, 6, 301, K, 30, 24, 2, neg_prob=0.2, cost="nonconvex")
    monkeypatch.setenv("ESDP_SHAPE", f"{R},{block}")
    monkeypatch.setenv("ESDP_EV", "tc")
    s = E.Solver([inst])
    s.autotune()
    info = s.launch_info()
    assert info["rows_per_thread"] == R and info["block"] == block
    assert info["ev"] == ("tcgen05" if K % 16 == 0 else "simt")
    V1 = s.solve_instances()[0]
    r = O.solve(inst, keep_EV=True, nthreads=NTHREADS)
    scale = _scale(r["V1"])
    assert_values(V1, r["V1"], scale)
    assert_policy(gpu_policies(s, inst), r["policy"], r["gap"], scale, inst=inst, EV=r["EV"])


VARIANT_CASES = [
    # R, block, K, modes: K = 63 or 64 take the fixed-stride variant, K = 13
    # (not a multiple of 4) the batch variant
    (4, 256, 64, 1), (8, 512, 64, 2), (9, 256, 63, 1), (10, 384, 64, 1), (12, 256, 63, 1),
    (4, 256, 13, 2), (6, 384, 13, 1), (8, 256, 13, 1), (9, 384, 13, 2), (10, 256, 13, 1),
    (12, 512, 13, 1),
]


@pytest.mark.parametrize("R,block,K,M", VARIANT_CASES,
                         ids=[f"R{c[0]}b{c[1]}K{c[2]}M{c[3]}" for c in VARIANT_CASES])
def test_rows_per_thread_in_every_kernel_variant(monkeypatch, R, block, K, M):
    """The rows-per-thread variants of the fixed-stride sweep (K = 63, 64)
    and of the batch sweep (K not a multiple of 4), pinned through
    ESDP_SHAPE, match the oracle's values and policies."""
    inst = I.random_instance(700 + R + K, 5, 301, K, 28, 26, M, neg_prob=0.2, cost="nonconvex")
    monkeypatch.setenv("ESDP_SHAPE", f"{R},{block}")
    s = E.Solver([inst])
    s.autotune()
    info = s.launch_info()
    assert info["rows_per_thread"] == R and info["block"] == block
    V1 = s.solve_instances()[0]
    r = O.solve(inst, keep_EV=True, nthreads=NTHREADS)
    scale = _scale(r["V1"])
    assert_values(V1, r["V1"], scale)
    assert_policy(gpu_policies(s, inst), r["policy"], r["gap"], scale, inst=inst, EV=r["EV"])


# ------------------------------------------------- EV contraction paths

EV_CASES = [
    # path pinned, K, modes
    ("tc", 16, 2), ("tc", 32, 1), ("tc", 64, 1), ("tc", 128, 2),
    ("mma", 8, 2), ("mma", 24, 1), ("mma", 40, 2), ("mma", 16, 1),
    ("simt", 16, 1), ("simt", 64, 2),
]
EV_NAMES = {"tc": "tcgen05", "mma": "mma.sync", "simt": "simt"}


@pytest.mark.parametrize("path,K,M", EV_CASES, ids=[f"{p}-K{k}-M{m}" for p, k, m in EV_CASES])
def test_ev_path_parity(monkeypatch, path, K, M):
    """Each unit that can contract EV (pinned through ESDP_EV on grids too
    small to pick it by themselves) gives the oracle's values, EV and
    policies."""
    monkeypatch.setenv("ESDP_EV", path)
    inst = I.random_instance(500 + K + M, 5, 301, K, 20, 24, M, neg_prob=0.2, cost="nonconvex")
    s = E.Solver([inst], keep_ev=True)
    assert s.launch_info()["ev"] == EV_NAMES[path]
    V1 = s.solve_instances()[0]
    r = O.solve(inst, keep_EV=True, nthreads=NTHREADS)
    scale = _scale(r["V1"])
    assert_values(V1, r["V1"], scale)
    assert_policy(gpu_policies(s, inst), r["policy"], r["gap"], scale, inst=inst, EV=r["EV"])
    ev = np.stack([s.expected_value(0, t) for t in range(1, inst.T + 1)])
    assert_values(ev, r["EV"], scale, "EV")


@pytest.mark.parametrize("N,K,M,want", [(5001, 64, 1, "tcgen05"), (5001, 72, 1, "mma.sync"),
                                        (2001, 64, 1, None), (5001, 56, 1, "simt"),
                                        (2001, 32, 1, "simt"), (1001, 128, 1, None),
                                        (301, 16, 2, "simt")])
def test_ev_path_follows_tile_work(N, K, M, want):
    """Without a pin the EV unit follows the contraction of a tile: with
    K >= 64 and at least 98,304 multiply-adds (rows x modes x K^2) tcgen05
    (K a multiple of 16) or mma.sync (K a multiple of 8), else FP32 SIMT."""
    inst = I.random_instance(600 + K, 3, N, K, 100, 100, M)
    s = E.Solver([inst])
    info = s.launch_info()
    work = info["rows_per_tile"] * M * K * K
    rule = "simt"
    if K >= 64 and work >= 98304:
        rule = "tcgen05" if K % 16 == 0 else ("mma.sync" if K % 8 == 0 else "simt")
    assert info["ev"] == rule
    if want is not None:  # else the tile size decides either way
        assert rule == want, f"tile of {info['rows_per_tile']} rows"
    s.close()


def test_autotune_discards_solve():
    """Tuning reuses the context's workspace: after it the results of the
    earlier solve are refused (ESDP_ESTATE) until the next solve, which
    gives the same objective."""
    inst = I.random_instance(61, 8, 200, 6, 12, 12, 1, neg_prob=0.2)
    inst.s0 = 90
    s = E.Solver([inst], keep_ev=True)
    s.solve_instances()
    J0 = s.grad(0, inst.mu0)[0][0]
    s.autotune()
    for call in (lambda: s.grad(0, inst.mu0), lambda: s.bid_curves(0, 1, 2),
                 lambda: s.policy(0, 1)):
        with pytest.raises(E.EsdpError) as ei:
            call()
        assert ei.value.code == E.ESDP_ESTATE
    s.solve_instances()
    assert s.grad(0, inst.mu0)[0][0] == pytest.approx(J0, rel=1e-6)


def test_gradient_in_batch_with_other_ev_path(monkeypatch):
    """The gradient of one asset of a batch re-sweeps it alone: with four
    assets its batch tile (40 rows x 64 states) contracts EV on tcgen05 while
    its own plan (about 8 rows) takes SIMT, so P is prepared again in the
    SIMT layout; the result equals the gradient from a context of that asset
    alone (same launch shape, same decisions) to float32 rounding."""
    insts = [I.random_instance(70 + j, 6, 1200, 64, 20, 20, 1, neg_prob=0.2) for j in range(4)]
    for inst in insts:
        inst.s0 = 600
    monkeypatch.setenv("ESDP_SHAPE", "8,512")
    s = E.Solver(insts)
    s.autotune()
    monkeypatch.delenv("ESDP_SHAPE")
    assert s.launch_info()["ev"] == "tcgen05"
    s.solve_instances()
    a = s.grad(0, insts[0].mu0, extra=True)
    one = E.Solver([insts[0]])
    assert one.launch_info()["ev"] == "simt"
    one.solve_instances()
    b = one.grad(0, insts[0].mu0, extra=True)
    for x, y in zip(a, b):
        x, y = np.asarray(x, np.float64), np.asarray(y, np.float64)
        assert np.abs(x - y).max() <= 1e-5 * max(np.abs(y).max(), 1e-30)


# ------------------------------------------------- packed bid curves

def test_bid_curves_packed_equal_padded():
    """Host and device packed forms hold exactly the padded rows' vertices and
    slopes (the envelope's last slope slot 0); a cap below the vertex total is
    rejected in host mode and truncates in device mode."""
    import torch
    inst = I.random_instance(24, 7, 333, 6, 25, 30, 2, neg_prob=0.3, cost="nonconvex")
    s, _ = solve_gpu(inst, keep_ev=True)
    n_bp, idx, slope = s.bid_curves(0, 2, inst.T + 1)
    off, pidx, psl = s.bid_curves_packed(0, 2, inst.T + 1)
    n = n_bp.reshape(-1)
    assert off[0] == 0 and np.array_equal(np.diff(off), n)
    rows_i, rows_s = idx.reshape(len(n), -1), slope.reshape(len(n), -1)
    for h in range(len(n)):
        a, b = off[h], off[h + 1]
        np.testing.assert_array_equal(pidx[a:b], rows_i[h, :n[h]])
        np.testing.assert_array_equal(psl[a:b - 1], rows_s[h, :n[h] - 1])
        assert psl[b - 1] == 0.0
    with pytest.raises(E.EsdpError) as ei:
        s.bid_curves_packed(0, 2, inst.T + 1, np.empty(len(n) + 1, np.int64),
                            np.empty(int(off[-1]) - 1, np.int32), np.empty(int(off[-1]) - 1, np.float32))
    assert ei.value.code == E.ESDP_EINVAL
    # device pointers
    cat = E.concat_inputs([inst])
    d = {k: torch.from_numpy(v).cuda() for k, v in cat.items()}
    ds = E.Solver([inst], device_ptrs=True, keep_ev=True)
    V1 = torch.empty(inst.n_modes * inst.N * inst.K, device="cuda")
    ds.solve(d["price"], d["trans"], d["cost"], d["terminal"], V1)
    doff = torch.empty(len(n) + 1, dtype=torch.int64, device="cuda")
    total = int(off[-1])
    di = torch.full((total,), -7, dtype=torch.int32, device="cuda")
    dsl = torch.empty(total, dtype=torch.float32, device="cuda")
    ds.bid_curves_packed(0, 2, inst.T + 1, doff, di, dsl)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(doff.cpu().numpy(), off)
    np.testing.assert_array_equal(di.cpu().numpy(), pidx)
    np.testing.assert_array_equal(dsl.cpu().numpy(), psl)
    short = torch.full((total - 5,), -7, dtype=torch.int32, device="cuda")
    shs = torch.empty(total - 5, dtype=torch.float32, device="cuda")
    ds.bid_curves_packed(0, 2, inst.T + 1, doff, short, shs)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(short.cpu().numpy(), pidx[:total - 5])
    ds.close()


# ------------------------------------------------- bids at a SoC state

@pytest.mark.parametrize("which", ["config2", "random"])
def test_bids_at_match_oracle(which):
    """esdp_bids_at against the oracle's markov_bids_at on the GPU's own EV:
    breakpoint counts and powers identical (the same double operations),
    prices identical after rounding to float32, prices non-decreasing."""
    if which == "config2":
        inst, T = I.config2(), 24            # the first day of 5-minute stages
    else:
        inst = I.random_instance(22, 6, 300, 5, 20, 35, 1, neg_prob=0.4, cost="nonconvex",
                                 eta=(0.85, 0.9))
        # stored energy left at the end costs $30/MWh: negative marginal values
        # in the last stages, where buying would pay more than selling
        x = np.arange(inst.N) * (inst.s_max / (inst.N - 1))
        inst.terminal[:] = (-30.0 * x).astype(np.float32)[None, :, None]
        T = inst.T
    s, V1 = solve_gpu(inst, keep_ev=True)
    n_bp, idx, _ = s.bid_curves(0, 1, T + 1)
    ev = np.stack([s.expected_value(0, t) for t in range(1, T + 1)])
    merged = 0
    for s_idx in (0, inst.N // 3, inst.N - 1):
        n_pts, p_mw, price = s.bids_at(0, 1, T + 1, s_idx, n_bp, idx)
        for t in range(T):
            for m in range(inst.n_modes):
                for k in range(inst.K):
                    xs, ps, prs = O.markov_bids_at(inst, ev[t, m, :, k], s_idx)
                    n = n_pts[t, m, k]
                    assert n == len(xs)
                    np.testing.assert_array_equal(p_mw[t, m, k, :n], ps)
                    np.testing.assert_array_equal(price[t, m, k, :n - 1],
                                                  np.asarray(prs, np.float64).astype(np.float32))
                    assert np.all(np.diff(price[t, m, k, :n - 1]) >= 0)
                    merged += 0.0 not in ps
    if which == "random":
        assert merged > 0   # negative marginal values: some curves merge the two sides


@pytest.mark.parametrize("N,Dd,Dc,modes", [
    (2, 1, 1, 1),        # two SoC points
    (40, 0, 6, 1),       # charge only: the window ends at s
    (40, 6, 0, 2),       # discharge only
    (33, 32, 32, 1),     # window wider than the grid on both sides
    (129, 3, 40, 2),     # asymmetric band
])
def test_bids_at_edge_windows(N, Dd, Dc, modes):
    inst = I.random_instance(40 + N, 4, N, 3, Dd, Dc, modes, neg_prob=0.3, cost="nonconvex",
                             eta=(0.88, 0.93))
    s, _ = solve_gpu(inst, keep_ev=True)
    n_bp, idx, _ = s.bid_curves(0, 1, inst.T + 1)
    ev = np.stack([s.expected_value(0, t) for t in range(1, inst.T + 1)])
    for s_idx in sorted({0, N // 2, N - 1}):
        n_pts, p_mw, price = s.bids_at(0, 1, inst.T + 1, s_idx, n_bp, idx)
        for t in range(inst.T):
            for m in range(inst.n_modes):
                for k in range(inst.K):
                    xs, ps, prs = O.markov_bids_at(inst, ev[t, m, :, k], s_idx)
                    n = n_pts[t, m, k]
                    assert n == len(xs) >= 1
                    np.testing.assert_array_equal(p_mw[t, m, k, :n], ps)
                    np.testing.assert_array_equal(price[t, m, k, :n - 1],
                                                  np.asarray(prs, np.float64).astype(np.float32))
                    if Dd == 0:
                        assert np.all(p_mw[t, m, k, :n] <= 0)   # nothing to sell
                    if Dc == 0:
                        assert np.all(p_mw[t, m, k, :n] >= 0)   # nothing to buy


def test_bids_at_rejects_invalid_vertex_lists():
    """Vertex lists that are not an envelope's (count out of range, unsorted,
    not spanning 0..N-1) give no bid (n_pts = 0) instead of reading outside
    the EV row; valid ones are unaffected."""
    inst = I.random_instance(26, 3, 80, 3, 5, 5, 1)
    s, _ = solve_gpu(inst, keep_ev=True)
    n_bp, idx, _ = s.bid_curves(0, 1, inst.T + 1)
    good = s.bids_at(0, 1, inst.T + 1, 40, n_bp, idx)[0]
    bad_n, bad_i = n_bp.copy(), idx.copy()
    bad_n[0, 0, 0] = inst.N + 5                     # count beyond the row
    bad_n[0, 0, 1] = 1                              # too few
    bad_i[1, 0, 0, :2] = [5, 3]                     # not starting at 0, unsorted
    bad_i[1, 0, 1, bad_n[1, 0, 1] - 1] = inst.N + 7  # last index outside the grid
    n_pts = s.bids_at(0, 1, inst.T + 1, 40, bad_n, bad_i)[0]
    assert n_pts[0, 0, 0] == 0 and n_pts[0, 0, 1] == 0
    assert n_pts[1, 0, 0] == 0 and n_pts[1, 0, 1] == 0
    np.testing.assert_array_equal(n_pts[2:], good[2:])


def test_bids_at_device_pointers_equal_host():
    import torch
    inst = I.random_instance(23, 5, 200, 4, 15, 15, 2, neg_prob=0.3)
    hs, _ = solve_gpu(inst, keep_ev=True)
    n_bp, idx, _ = hs.bid_curves(0, 1, inst.T + 1)
    ref = hs.bids_at(0, 1, inst.T + 1, 77, n_bp, idx)
    cat = E.concat_inputs([inst])
    d = {k: torch.from_numpy(v).cuda() for k, v in cat.items()}
    ds = E.Solver([inst], device_ptrs=True, keep_ev=True)
    V1 = torch.empty(inst.n_modes * inst.N * inst.K, device="cuda")
    ds.solve(d["price"], d["trans"], d["cost"], d["terminal"], V1)
    sh = (inst.T, inst.n_modes, inst.K)
    dn = torch.empty(sh, dtype=torch.int32, device="cuda")
    di = torch.empty(sh + (inst.N,), dtype=torch.int32, device="cuda")
    dsl = torch.empty(sh + (inst.N,), dtype=torch.float32, device="cuda")
    ds.bid_curves(0, 1, inst.T + 1, dn, di, dsl)
    n_pts = torch.empty(sh, dtype=torch.int32, device="cuda")
    p_mw = torch.empty(sh + (inst.A,), dtype=torch.float64, device="cuda")
    price = torch.empty(sh + (inst.A,), dtype=torch.float32, device="cuda")
    ds.bids_at(0, 1, inst.T + 1, 77, dn, di, n_pts, p_mw, price)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(n_pts.cpu().numpy(), ref[0])
    n = ref[0]
    for i in np.ndindex(*sh):
        np.testing.assert_array_equal(p_mw.cpu().numpy()[i][:n[i]], ref[1][i][:n[i]])
        np.testing.assert_array_equal(price.cpu().numpy()[i][:n[i] - 1], ref[2][i][:n[i] - 1])
    ds.close()


# ------------------------------------------------- torch.autograd.Function

def test_autograd_objective_matches_oracle_adjoint():
    import torch
    from paper_2511_15629_b300.autograd import StorageObjective
    inst = I.random_instance(53, 6, 25, 3, 3, 3, 1, neg_prob=0.2, cost="linear")
    inst.s0 = 12
    f = StorageObjective(inst)
    dev = f.device
    price = torch.tensor(inst.price, device=dev, requires_grad=True)
    trans = torch.tensor(inst.trans, device=dev, requires_grad=True)
    eta_c = torch.tensor(inst.eta_c, dtype=torch.float64, requires_grad=True)
    eta_d = torch.tensor(inst.eta_d, dtype=torch.float64, requires_grad=True)
    cost = torch.tensor(inst.cost, device=dev, requires_grad=True)
    terminal = torch.tensor(inst.terminal, device=dev, requires_grad=True)
    mu0 = torch.tensor(inst.mu0, device=dev, requires_grad=True)
    J = f(price, trans, eta_c, eta_d, cost=cost, terminal=terminal, mu0=mu0)
    # another solve in between: backward must recompute the first one
    J_other = f(price.detach() * 2, trans.detach())
    J.backward()
    r = O.solve(inst, keep_V=True, nthreads=NTHREADS)
    assert float(J.detach()) == pytest.approx(O.objective(inst, r["V1"]), rel=VTOL)
    assert float(J_other) != pytest.approx(float(J.detach()), rel=1e-3)
    occ = O.occupancy(inst, r["policy"], r["V"])
    for g, key in ((price.grad, "d_price"), (trans.grad, "d_trans"),
                   (eta_c.grad, "d_eta_c"), (eta_d.grad, "d_eta_d"), (cost.grad, "d_cost"),
                   (terminal.grad, "d_terminal"), (mu0.grad, "d_mu0")):
        ref = np.atleast_1d(occ[key])
        got = g.detach().cpu().numpy().astype(np.float64).reshape(ref.shape)
        err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-12)
        assert err <= 1e-4, f"{key}: rel error {err:.3e}"
    # central differences of the GPU forward in eta_c (float32 values: the
    # quotient carries ~1e-7 |J| / h of noise)
    h = 1e-4
    with torch.no_grad():
        jp = float(f(price, trans, eta_c + h, eta_d))
        jm = float(f(price, trans, eta_c - h, eta_d))
    fd = (jp - jm) / (2 * h)
    assert fd == pytest.approx(float(eta_c.grad), rel=2e-2, abs=1e-7 * abs(float(J.detach())) / h)


def test_price_gradient_vs_gpu_central_differences():
    """dJ/dprice from the occupancy adjoint against central differences of
    the GPU's own forward solve (h = 1e-3 $/MWh) on a tie-free instance (every
    top-two gap far above what a step of h can move, h max|e_a|): the six
    stage prices with the largest sensitivity, the quotient's float32 noise
    (about 1e-7 |J| / h) allowed for as in the efficiency check."""
    make = lambda: I.random_instance(61, 4, 60, 2, 4, 4, 1, neg_prob=0.0, cost="linear",
                                     s_max=59.0)
    inst = make()
    inst.s0 = 30
    h = 1e-3
    r = O.solve(inst, keep_V=True, nthreads=NTHREADS)
    e_max = max(inst.D_dis * inst.delta * inst.eta_d, inst.D_chg * inst.delta / inst.eta_c)
    assert r["gap"][np.isfinite(r["gap"])].min() > 20 * h * e_max, "the seed must be tie-free"
    s, _ = solve_gpu(inst)
    J0, dp = s.grad(0, inst.mu0)[:2]
    dp = np.asarray(dp, np.float64).reshape(inst.T, inst.K)
    order = np.argsort(-np.abs(dp).ravel())[:6]
    for flat in order:
        t, k = np.unravel_index(flat, dp.shape)
        vals = []
        for sign in (1.0, -1.0):
            pert = make()
            pert.s0 = 30
            pert.price = pert.price.astype(np.float64)
            pert.price[t, k] += sign * h
            pert.price = pert.price.astype(np.float32)
            step = float(pert.price[t, k]) - float(inst.price[t, k])   # the float32 step taken
            sp, V1 = solve_gpu(pert)
            vals.append((float(np.dot(inst.mu0.astype(np.float64), V1[0, inst.s0, :])), step))
        fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
        noise = 1e-7 * abs(float(J0[0])) / h
        assert fd == pytest.approx(dp[t, k], rel=2e-2, abs=noise), (t, k, fd, dp[t, k])


def test_transition_gradient_vs_gpu_central_differences():
    """dJ/dP from the occupancy adjoint against central differences of the
    GPU's own forward solve: one transition entry P_t[k][k2] moved by +-h
    (h = 1e-4, the float32 step actually taken) on a tie-free instance (every
    top-two gap far above what the step can move, h max|V|), for the four
    entries with the largest sensitivity; the quotient's float32 noise
    allowed for as in the price check."""
    make = lambda: I.random_instance(63, 4, 60, 3, 4, 4, 1, neg_prob=0.0, cost="linear",
                                     s_max=59.0)
    inst = make()
    inst.s0 = 30
    h = 1e-4
    r = O.solve(inst, keep_V=True, nthreads=NTHREADS)
    v_max = float(np.abs(r["V"]).max())
    assert r["gap"][np.isfinite(r["gap"])].min() > 20 * h * v_max, "the seed must be tie-free"
    s, _ = solve_gpu(inst)
    J0, _, dt = s.grad(0, inst.mu0)[:3]
    dt = np.asarray(dt, np.float64).reshape(inst.T, inst.K, inst.K)
    order = np.argsort(-np.abs(dt).ravel())[:4]
    for flat in order:
        t, k, k2 = np.unravel_index(flat, dt.shape)
        vals = []
        for sign in (1.0, -1.0):
            pert = make()
            pert.s0 = 30
            p64 = pert.trans.astype(np.float64)
            p64[t, k, k2] += sign * h
            pert.trans = p64.astype(np.float32)
            step = float(pert.trans[t, k, k2]) - float(inst.trans[t, k, k2])
            _, V1 = solve_gpu(pert)
            vals.append((float(np.dot(inst.mu0.astype(np.float64), V1[0, inst.s0, :])), step))
        fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
        noise = 1e-7 * abs(float(J0[0])) / h
        assert fd == pytest.approx(dt[t, k, k2], rel=2e-2, abs=noise), (t, k, k2, fd, dt[t, k, k2])


def test_autograd_checkpointed_int16():
    import torch
    from paper_2511_15629_b300.autograd import StorageObjective
    inst = I.random_instance(54, 40, 120, 5, 9, 9, 2, neg_prob=0.2, switch_cost=3.0)
    inst.s0 = 60
    inst.ckpt_every = 7
    inst.policy_bytes = 2
    f = StorageObjective(inst)
    price = torch.tensor(inst.price, device=f.device, requires_grad=True)
    trans = torch.tensor(inst.trans, device=f.device, requires_grad=True)
    sw = torch.tensor(inst.switch_cost, dtype=torch.float64, requires_grad=True)
    f(price, trans, switch_cost=sw).backward()
    s, _ = solve_gpu(inst)
    J, dp, dt, de, dco, dsw, dterm, dmu = s.grad(0, inst.mu0, extra=True)
    assert float(sw.grad) == pytest.approx(dsw[0], rel=1e-6, abs=1e-12)
    # same adjoint through the autograd wrapper and through esdp_grad; the
    # occupancy scatter adds in fixed point and every other sum runs in a
    # fixed order, so the two agree (the tolerance only allows for the
    # autograd wrapper's own float32 conversions)
    np.testing.assert_allclose(price.grad.cpu().numpy(), dp, rtol=1e-6, atol=1e-6 * np.abs(dp).max())
    np.testing.assert_allclose(trans.grad.cpu().numpy(), dt, rtol=1e-6, atol=1e-6 * np.abs(dt).max())
