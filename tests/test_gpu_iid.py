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


def test_iid_tiles_taller_than_one_pass():
    """S = 10001 on 148 SMs gives 68-row tiles while 64 samples per row fill
    only 64 rows per pass of the block: rows are taken in two passes."""
    prob = I.iid_problem(10, 6, 10001, 64, 1000.0)
    _check_values(E.solve_iid(prob), _oracle(prob)[0])
