"""GPU parity of the stagewise-independent path (esdp_solve_iid) against the
oracle's literal Algorithm 1 (FP64, eq. 13 action grid with interpolated end
points).  Tolerances as for the Markov sweep: values within 1e-5 max|V_0|,
argmax actions identical wherever the oracle's top-two gap is at least
1e-6 max|V_0|."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_15629_b300 import esdp as E
from paper_2511_15629_b300 import instances as I

pytestmark = pytest.mark.gpu

VTOL = 1e-5
GAPTOL = 1e-6


def _oracle(prob, keep_policy=False):
    return O.paper_alg1(prob.s_max, prob.delta, prob.p_max, prob.eta, prob.lam_hat, prob.pi_hat,
                        terminal=prob.terminal, tau=prob.tau, keep_policy=keep_policy)


def _check_values(V0, ref):
    scale = max(np.abs(ref).max(), 1.0)
    err = np.abs(V0.astype(np.float64) - ref).max() / scale
    assert err <= VTOL, f"max rel error {err:.3e}"
    return scale


@pytest.mark.parametrize("case", [
    dict(seed=1, T=30, S=81, R=12, hours=4.0),                       # end points off the grid
    dict(seed=2, T=40, S=41, R=7, hours=4.0, weights="dirichlet"),    # P = 22 (Table I row 1)
    dict(seed=3, T=25, S=101, R=33, hours=2.0, terminal=True),        # terminal value, ragged groups
    dict(seed=4, T=20, S=61, R=5, hours=3.0, eta=1.0),                # recombining: end points on grid
    dict(seed=5, T=16, S=201, R=200, hours=2.0),                      # R = 200 samples (the paper's)
])
def test_iid_values_match_algorithm1(case):
    prob = I.iid_problem(**case)
    V0 = E.solve_iid(prob)
    ref = _oracle(prob)[0]
    _check_values(V0, ref)


def test_iid_quarter_hour_stages():
    prob = I.iid_problem(6, 24, 121, 9, 3.0)
    prob.tau = 0.25
    _check_values(E.solve_iid(prob), _oracle(prob)[0])


@pytest.mark.parametrize("pb", [4, 2])
def test_iid_policy_matches_outside_near_ties(pb):
    prob = I.iid_problem(7, 12, 81, 10, 4.0, weights="dirichlet")
    V0, pol = E.solve_iid(prob, policy_bytes=pb)
    V, ref_pol, gap = _oracle(prob, keep_policy=True)
    scale = _check_values(V0, V[0])
    decided = gap >= GAPTOL * scale
    bad = (pol.astype(np.int64) != ref_pol) & decided
    assert not bad.any(), f"{int(bad.sum())} policy mismatches outside near-ties"
    assert decided.mean() > 0.5


def test_iid_table3_launch_shape_sample():
    """The 4 h / S = 401 / P = 203 Table III case with the paper's R = 200
    samples on a 48-stage horizon: the launch configuration of the full
    benchmark (rows per tile, halo reach), checked against Algorithm 1."""
    prob = I.table3_problem(3, T=48)
    assert len(E.iid_actions(prob)) == 203
    _check_values(E.solve_iid(prob), _oracle(prob)[0])


def test_iid_device_pointers_and_value_identity():
    torch = pytest.importorskip("torch")
    prob = I.iid_problem(8, 20, 101, 16, 4.0, terminal=True)
    host = E.solve_iid(prob)
    lam = torch.from_numpy(prob.lam_hat).cuda()
    pi = torch.from_numpy(prob.pi_hat).cuda()
    term = torch.from_numpy(prob.terminal).cuda()
    V0 = torch.empty(prob.S, device="cuda")
    E.solve_iid(prob, V0, device=True, lam_hat=lam, pi_hat=pi, terminal=term)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(V0.cpu().numpy(), host)


def test_iid_equals_markov_sweep_on_recombining_grid():
    """eta = 1 and p_max a multiple of delta: no end-point interpolation, so
    Algorithm 1 is the Markov DP with the rank-1 transitions P_t = 1 pi_{t+1}^T
    and the esdp_solve sweep must give the same V_0 (up to float32)."""
    T, S, R, hours = 12, 41, 6, 4.0
    prob = I.iid_problem(9, T, S, R, hours, eta=1.0)
    V0 = E.solve_iid(prob)
    # the same problem as a Markov instance: K = R states, shifts -D..D
    D = int(round(prob.p_max / prob.delta))
    inst = I.random_instance(9, T, S, R, D, D, 1, cost="zero", terminal="zero",
                             eta=(1.0, 1.0), s_max=prob.s_max, tau=1.0)
    inst.price = np.ascontiguousarray(prob.lam_hat)
    pis = np.concatenate([prob.pi_hat, prob.pi_hat[-1:]], axis=0)
    inst.trans = np.ascontiguousarray(np.broadcast_to(pis[1:, None, :], (T, R, R)).copy())
    s = E.Solver([inst])
    V1 = s.solve_instances()[0]                       # V_1[0][s][k]
    Vm = V1[0].astype(np.float64) @ prob.pi_hat[0].astype(np.float64)
    scale = max(np.abs(Vm).max(), 1.0)
    assert np.abs(V0 - Vm).max() / scale <= 2e-5


@pytest.mark.parametrize("S", [10001, 7400])
def test_iid_tiles_taller_than_one_pass(S):
    """Tall tiles with 64 samples per row: S = 10001 gives 68-row tiles
    (10 samples per thread take them in one pass of the block, 8 would need
    two), S = 7400 gives 50-row tiles (8 samples per thread, one pass; 6
    would need two).  The samples-per-thread variants are chosen by work per
    thread, so these shapes exercise the ones the small tests do not."""
    prob = I.iid_problem(10, 6, S, 64, 1000.0)
    V0, pol = E.solve_iid(prob, policy_bytes=4)
    V, ref_pol, gap = _oracle(prob, keep_policy=True)
    scale = _check_values(V0, V[0])
    decided = gap >= GAPTOL * scale
    assert not ((pol.astype(np.int64) != ref_pol) & decided).any()


# ------------------------------------------------ bid curves and clearing

def _device_values(prob):
    import torch
    lam = torch.from_numpy(prob.lam_hat).cuda()
    pi = torch.from_numpy(prob.pi_hat).cuda()
    V0 = torch.empty(prob.S, device="cuda")
    V_all = torch.empty((prob.T + 1, prob.S), device="cuda")
    E.solve_iid(prob, V0, device=True, lam_hat=lam, pi_hat=pi, V_all=V_all)
    torch.cuda.synchronize()
    return V0, V_all


def test_iid_kept_values_match_algorithm1():
    prob = I.iid_problem(12, 20, 81, 9, 4.0, terminal=True)
    V0, pol, V_all = E.solve_iid(prob, policy_bytes=4, keep_values=True)
    np.testing.assert_array_equal(V_all[0], V0)
    ref = _oracle(prob)
    scale = max(np.abs(ref).max(), 1.0)
    assert np.abs(V_all.astype(np.float64) - ref).max() / scale <= VTOL


def test_iid_bid_curves_bit_exact():
    """Vertices identical to the oracle's envelope on the GPU's own values
    (same double predicate), prices to float32, monotone bids."""
    prob = I.iid_problem(13, 10, 61, 8, 3.0, neg_prob=0.3)
    _, V_all = _device_values(prob)
    n_bp, act, price = E.iid_bids(prob, V_all, 1, prob.T + 1)
    n_bp, act, price = n_bp.cpu().numpy(), act.cpu().numpy(), price.cpu().numpy()
    V = V_all.cpu().numpy()
    non_concave = 0
    for t in range(1, prob.T + 1):
        for s in range(prob.S):
            idx, pr = O.paper_bids(prob.S, prob.s_max, prob.p_max, prob.eta, prob.tau, V[t], s)
            n = n_bp[t - 1, s]
            assert n == len(idx)
            np.testing.assert_array_equal(act[t - 1, s, :n], idx)
            np.testing.assert_allclose(price[t - 1, s, :n - 1], pr, rtol=1e-6, atol=1e-6)
            assert np.all(np.diff(price[t - 1, s, :n - 1]) >= 0)
            p, f = O._shifts(prob.S, prob.s_max, prob.p_max, prob.eta, prob.tau)
            feas = sum(1 for a in range(len(p)) if -1e-9 <= s + f[a] <= prob.S - 1 + 1e-9)
            non_concave += n < feas
    assert non_concave > 0   # negative prices make some U non-concave: convexification acts


def test_iid_clearing_matches_oracle():
    import torch
    prob = I.iid_problem(14, 24, 41, 6, 4.0, neg_prob=0.2)
    _, V_all = _device_values(prob)
    rng = np.random.default_rng(5)
    lam = (prob.lam_hat.mean(axis=1)[None, :] * rng.lognormal(0.0, 0.4, size=(16, prob.T))
           - 5.0).astype(np.float32)
    rev, s_end, act = E.iid_clear(prob, V_all, torch.from_numpy(lam).cuda(), 2.0)
    rev, s_end, act = rev.cpu().numpy(), s_end.cpu().numpy(), act.cpu().numpy()
    V = V_all.cpu().numpy()
    for i in range(lam.shape[0]):
        r, z, a = O.paper_clear(prob.S, prob.s_max, prob.p_max, prob.eta, prob.tau, V, lam[i], 2.0)
        np.testing.assert_array_equal(act[i], a)
        assert rev[i] == pytest.approx(r, rel=1e-12, abs=1e-9)
        assert s_end[i] == pytest.approx(z, abs=1e-9)


@pytest.mark.parametrize("case", ["endpoints", "ties"])
def test_iid_clearing_exact_on_hard_paths(case):
    """The float32 enclosure in the clearing kernel must never change a
    decision: 64 paths with fractional end-point shifts and prices swinging
    from -60 to 150 (the SoC reaches both ends of the grid), and a case where
    every action ties (zero prices, zero values: the smallest feasible index
    is cleared at every stage)."""
    import torch
    prob = I.iid_problem(16, 30, 61, 5, 3.0, p_max=1.3, neg_prob=0.3)
    if case == "endpoints":
        _, V_all = _device_values(prob)
        rng = np.random.default_rng(23)
        lam = rng.uniform(-60.0, 150.0, size=(64, prob.T)).astype(np.float32)
        s0 = 1.5
    else:
        V_all = torch.zeros((prob.T + 1, prob.S), device="cuda")
        lam = np.zeros((8, prob.T), np.float32)
        s0 = 0.0
    rev, s_end, act = E.iid_clear(prob, V_all, torch.from_numpy(lam).cuda(), s0)
    rev, s_end, act = rev.cpu().numpy(), s_end.cpu().numpy(), act.cpu().numpy()
    V = V_all.cpu().numpy()
    ends = 0
    for i in range(lam.shape[0]):
        r, z, a = O.paper_clear(prob.S, prob.s_max, prob.p_max, prob.eta, prob.tau, V, lam[i], s0)
        np.testing.assert_array_equal(act[i], a)
        assert rev[i] == pytest.approx(r, rel=1e-12, abs=1e-9)
        assert s_end[i] == pytest.approx(z, abs=1e-9)
    if case == "endpoints":
        p, f = O._shifts(prob.S, prob.s_max, prob.p_max, prob.eta, prob.tau)
        assert any(abs(x - round(x)) > 1e-6 for x in f)   # fractional end-point shifts
        assert (act == 0).any() and (act == len(p) - 1).any()


def test_iid_clearing_monte_carlo_reproduces_value():
    """Price paths drawn from the model's own samples (eta = 1: every action
    on the grid): the mean cleared revenue is V_0(s0) within 3 standard
    errors."""
    import torch
    prob = I.iid_problem(15, 48, 81, 12, 4.0, eta=1.0, weights="dirichlet")
    V0, V_all = _device_values(prob)
    rng = np.random.default_rng(9)
    n = 20000
    pi = prob.pi_hat.astype(np.float64)
    cum = np.cumsum(pi / pi.sum(axis=1, keepdims=True), axis=1)
    u = rng.random((n, prob.T))
    k = (u[:, :, None] > cum[None, :, :]).sum(axis=2).clip(0, prob.R - 1)
    lam = prob.lam_hat[np.arange(prob.T)[None, :], k].astype(np.float32)
    rev, _, _ = E.iid_clear(prob, V_all, torch.from_numpy(lam).cuda(), 2.0, keep_actions=False)
    rev = rev.cpu().numpy()
    se = rev.std(ddof=1) / math.sqrt(n)
    target = float(V0.cpu().numpy()[int(round(2.0 / prob.delta))])
    assert abs(rev.mean() - target) <= 3 * se, (rev.mean(), target, se)


@pytest.mark.parametrize("kw", [
    dict(S=2, R=1, hours=1.0),                         # two SoC points, one sample
    dict(S=11, R=3, hours=1.0, p_max=0.03),            # p_max below one SoC step: P = 3
    dict(S=21, R=4, hours=0.5, p_max=2.0),             # end points beyond the whole range
    dict(S=301, R=9, hours=30.0, p_max=5.0),           # wide action grid, halo over many tiles
    dict(S=21, R=4096, hours=2.0),                     # the most samples per stage
])
def test_iid_edge_shapes(kw):
    hours = kw.pop("hours")
    p_max = kw.pop("p_max", 1.0)
    prob = I.iid_problem(30, 12, kw["S"], kw["R"], hours, p_max=p_max)
    P = len(E.iid_actions(prob))
    assert P >= 3
    V0, pol = E.solve_iid(prob, policy_bytes=4)
    V, ref_pol, gap = _oracle(prob, keep_policy=True)
    scale = _check_values(V0, V[0])
    decided = gap >= GAPTOL * scale
    assert not ((pol.astype(np.int64) != ref_pol) & decided).any()
