"""Pins of the FP64 oracle against things other than itself (CPU only).

* Table I / Table III action and grid counts (golden files);
* exhaustive enumeration of every non-anticipative policy on tiny trees;
* an independent longest path over the (time x SoC [x mode]) DAG for K = 1;
* one-stage closed forms of eq. 5 with a linear terminal value;
* Algorithm 1 taken literally (interpolated end points) against the Markov
  oracle and against closed forms;
* DP <= LP (SciPy HiGHS) with the gap shrinking as delta -> 0 (Sec. V-A);
* invariants (V >= 0 with free idling, concavity in SoC, base case);
* Monte Carlo forward simulation within 3 standard errors;
* the occupancy identity J = sum_t E[r_t] + E[V_{T+1}] and central finite
  differences of the gradients.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_15629_b300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid_energy(inst, a):
    """Grid-side energy of shifting the SoC by d = a - D_dis grid steps,
    written from the paper's power variables: discharging p MW for one
    stage removes p/eta_d of stored energy (eq. 3b), charging p MW adds
    eta_c p (eq. 3b)."""
    d = a - inst.D_dis
    stored = d * inst.delta            # change of stored energy (MWh)
    if d < 0:
        return (-stored) * inst.eta_d   # p^d with p^d / eta_d = -stored
    if d > 0:
        return -(stored / inst.eta_c)   # -p^c with eta_c p^c = stored
    return 0.0


def _load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


# ---------------------------------------------------------------- Table pins

def test_table1_action_counts():
    eta = math.sqrt(0.85)
    for delta, P in _load_golden("table1_action_counts.txt"):
        p_hat, n_c, n_d = O.paper_action_grid(1.0, delta, eta)
        assert len(p_hat) == int(P), (delta, len(p_hat), P)
        assert n_c + n_d + 1 == int(P)


def test_table3_grid_sizes():
    eta = math.sqrt(0.85)
    for dur, delta, S, P in _load_golden("table3_grid_sizes.txt"):
        assert int(round(dur / delta)) + 1 == int(S)
        p_hat, _, _ = O.paper_action_grid(1.0, delta, eta)
        assert len(p_hat) == int(P)


def test_action_grid_structure():
    """eq. 13: charge actions are -j delta/eta plus -p_max, discharge
    actions j delta eta plus p_max; F maps the interior to integer shifts."""
    eta, delta, p_max = math.sqrt(0.85), 0.1, 1.0
    p_hat, n_c, n_d = O.paper_action_grid(p_max, delta, eta)
    F = O.paper_F(p_hat, eta)
    assert p_hat[0] == -p_max and p_hat[-1] == p_max
    assert np.all(np.diff(p_hat) > 0)
    interior = F[1:-1] / delta
    assert np.allclose(interior, np.round(interior), atol=1e-9)
    assert np.isclose(F[0], p_max * eta) and np.isclose(F[-1], -p_max / eta)
    # charging raises the SoC, discharging lowers it (eq. 2)
    assert np.all(F[p_hat < 0] > 0) and np.all(F[p_hat > 0] < 0)


# ------------------------------------------------- exhaustive policy search

def _enumerate_policies(inst):
    """Best expected value over every non-anticipative policy.

    A policy assigns an action to every price history (k_1..k_t), t <= T.
    Its value is the probability-weighted sum over complete price paths of
    the stage payoffs plus the terminal value; policies that leave the SoC
    range on any path are discarded.  The charge->discharge switch cost is
    charged from the action history itself (discharge whose most recent
    non-idle predecessor was a charge)."""
    T, K, A = inst.T, inst.K, inst.A
    price = inst.price.astype(np.float64)
    trans = inst.trans.astype(np.float64)
    cost = inst.cost.astype(np.float64)
    term = inst.terminal.astype(np.float64)
    mu0 = inst.mu0.astype(np.float64)
    nodes = []
    for t in range(1, T + 1):
        nodes += list(itertools.product(range(K), repeat=t))
    node_id = {h: i for i, h in enumerate(nodes)}

    def policy_value(assign):
        # walk the whole scenario tree under one fixed policy; the payoff of
        # a stage is weighted by the probability of the price history that
        # reaches it (float32 rows need not sum to exactly one)
        total = 0.0
        stack = [((k,), inst.s0, False, mu0[k]) for k in range(K)]
        while stack:
            h, s, last_charge, pr = stack.pop()
            t = len(h)
            a = assign[node_id[h]]
            d = a - inst.D_dis
            s2 = s + d
            if s2 < 0 or s2 > inst.N - 1:
                return None
            r = price[t - 1, h[-1]] * _grid_energy(inst, a) - cost[a]
            if inst.n_modes == 2 and d < 0 and last_charge:
                r -= inst.switch_cost
            lc = True if d > 0 else (False if d < 0 else last_charge)
            total += pr * r
            for k2 in range(K):
                p2 = pr * trans[t - 1, h[-1], k2]
                if t < T:
                    stack.append((h + (k2,), s2, lc, p2))
                else:
                    mode = 1 if (inst.n_modes == 2 and lc) else 0
                    total += p2 * term[mode, s2, k2]
        return total

    best = -math.inf
    for assign in itertools.product(range(A), repeat=len(nodes)):
        v = policy_value(assign)
        if v is not None:
            best = max(best, v)
    return best


@pytest.mark.parametrize("T,K,N,Dd,Dc,modes,seed", [
    (2, 2, 5, 1, 1, 1, 1), (2, 2, 5, 1, 1, 2, 2), (2, 2, 4, 2, 1, 1, 3),
    (3, 1, 5, 1, 1, 2, 4), (4, 1, 6, 1, 1, 1, 5), (3, 2, 3, 1, 0, 1, 6),
    (2, 2, 6, 2, 2, 2, 7),
])
def test_exhaustive_policy_enumeration(T, K, N, Dd, Dc, modes, seed):
    inst = I.random_instance(seed, T, N, K, Dd, Dc, modes, neg_prob=0.3, switch_cost=9.0,
                             cost="nonconvex")
    for s0 in sorted({0, N // 2, N - 1}):
        inst.s0 = s0
        ref = _enumerate_policies(inst)
        r = O.solve(inst)
        assert O.objective(inst, r["V1"]) == pytest.approx(ref, rel=1e-12, abs=1e-9)


# ---------------------------------------------- longest path over the DAG

def _dag_longest(inst):
    """K = 1: V_1[m=0][s] for every s as a longest path through the DAG with
    nodes (t, s, m) for t = 1..T+1, built as an explicit edge list and
    processed in Kahn topological order from a super source per start."""
    assert inst.K == 1
    T, N, A, M = inst.T, inst.N, inst.A, inst.n_modes
    price = inst.price.astype(np.float64)[:, 0]
    cost = inst.cost.astype(np.float64)
    nid = {}
    for t in range(1, T + 2):
        for s in range(N):
            for m in range(M):
                nid[(t, s, m)] = len(nid)
    sink = len(nid)
    edges = []
    for (t, s, m), u in nid.items():
        if t == T + 1:
            edges.append((u, sink, float(inst.terminal[m, s, 0])))
            continue
        for a in range(A):
            d = a - inst.D_dis
            s2 = s + d
            if not 0 <= s2 < N:
                continue
            r = price[t - 1] * _grid_energy(inst, a) - cost[a]
            m2 = m
            if M == 2:
                if d < 0 and m == 1:
                    r -= inst.switch_cost
                m2 = 0 if d < 0 else (1 if d > 0 else m)
            edges.append((u, nid[(t + 1, s2, m2)], r))
    n = sink + 1
    out = [[] for _ in range(n)]
    indeg = [0] * n
    for u, v, w in edges:
        out[u].append((v, w))
        indeg[v] += 1
    order = []
    q = [u for u in range(n) if indeg[u] == 0]
    while q:
        u = q.pop()
        order.append(u)
        for v, _ in out[u]:
            indeg[v] -= 1
            if indeg[v] == 0:
                q.append(v)
    assert len(order) == n
    res = []
    for s0 in range(N):
        dist = [-math.inf] * n
        dist[nid[(1, s0, 0)]] = 0.0
        for u in order:
            if dist[u] == -math.inf:
                continue
            for v, w in out[u]:
                if dist[u] + w > dist[v]:
                    dist[v] = dist[u] + w
        res.append(dist[sink])
    return np.array(res)


@pytest.mark.parametrize("T,N,Dd,Dc,modes,seed", [
    (6, 9, 2, 3, 1, 11), (8, 12, 3, 3, 2, 12), (5, 7, 6, 1, 1, 13), (7, 10, 2, 2, 2, 14),
])
def test_deterministic_longest_path(T, N, Dd, Dc, modes, seed):
    inst = I.random_instance(seed, T, N, 1, Dd, Dc, modes, neg_prob=0.3, switch_cost=6.0,
                             cost="nonconvex")
    r = O.solve(inst)
    np.testing.assert_allclose(r["V1"][0, :, 0], _dag_longest(inst), rtol=1e-12, atol=1e-9)


# ----------------------------------------------------- one-stage closed form

@pytest.mark.parametrize("lam,v", [(50.0, 30.0), (20.0, 30.0), (31.0, 30.0), (-15.0, 10.0),
                                   (-5.0, -3.0), (40.0, 40.0 * 0.9)])
def test_one_stage_closed_form(lam, v):
    """T = 1, K = 1, zero cost, terminal v $/MWh of stored energy.
    Discharging x MWh of storage earns lam*eta_d*x - v*x, charging x earns
    v*x - lam*x/eta_c (the payoff of eq. 5 with eq. 2); both are linear in
    x, so the optimum is idle or the largest feasible shift."""
    N, Dd, Dc = 21, 4, 6
    inst = I.random_instance(0, 1, N, 1, Dd, Dc, 1, terminal="linear", cost="zero",
                             eta=(0.8, 0.9))
    inst.price[:] = np.float32(lam)
    delta = inst.delta
    soc = np.arange(N) * delta
    inst.terminal[:] = (np.float32(v) * soc.astype(np.float32))[None, :, None].astype(np.float32)
    term = inst.terminal[0, :, 0].astype(np.float64)
    vv = float(np.float32(v))
    lam32 = float(np.float32(lam))
    r = O.solve(inst)
    for s in range(N):
        xd = min(Dd, s) * delta
        xc = min(Dc, N - 1 - s) * delta
        ref = term[s] + max(0.0, xd * (lam32 * inst.eta_d - vv), xc * (vv - lam32 / inst.eta_c))
        assert r["V1"][0, s, 0] == pytest.approx(ref, rel=1e-6, abs=1e-6), s


def test_one_stage_closed_form_detects_swapped_efficiencies():
    """Planted mistake: an oracle run with eta_c and eta_d exchanged must
    disagree with the closed form (so the pin above can see that error)."""
    N, Dd, Dc = 21, 4, 6
    inst = I.random_instance(0, 1, N, 1, Dd, Dc, 1, terminal="zero", cost="zero", eta=(0.8, 0.9))
    inst.price[:] = np.float32(50.0)
    good = O.solve(inst)["V1"][0, N - 1, 0]
    bad = O.solve(inst, eta_c=inst.eta_d, eta_d=inst.eta_c)["V1"][0, N - 1, 0]
    ref = Dd * inst.delta * 50.0 * inst.eta_d
    assert good == pytest.approx(ref, rel=1e-9)
    assert abs(bad - ref) > 1e-3


# ------------------------------------------------------- Algorithm 1 literal

def _recombining_iid(seed, T, R):
    """eta = 0.5, delta = 1/8, p_max = 1/2, s_max = 2: p_max eta / delta = 2
    and p_max / (delta eta) = 8 are integers, so the end points of eq. 13 fall
    on the grid and Alg. 1 needs no interpolation."""
    inst = I.iid_instance(seed, T, 17, R, 8, 2, cost="zero", terminal="zero", eta=(0.5, 0.5),
                          s_max=2.0)
    return inst


@pytest.mark.parametrize("seed,T,R", [(21, 5, 3), (22, 9, 6), (23, 3, 1)])
def test_alg1_literal_equals_markov_oracle(seed, T, R):
    inst = _recombining_iid(seed, T, R)
    pis = inst.meta["pi_hat"].astype(np.float64)
    lam = inst.price.astype(np.float64)
    Vhat = O.paper_alg1(2.0, 0.125, 0.5, 0.5, lam, pis[:T])
    r = O.solve(inst, keep_EV=True)
    # V_hat_{t} (paper) = EV_t (Markov) for t = 1..T-1 ... and V_hat_0 = J(s)
    for t in range(1, T):
        np.testing.assert_allclose(Vhat[t], r["EV"][t - 1, 0, :, 0], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(Vhat[0], r["V1"][0] @ inst.mu0.astype(np.float64), rtol=1e-12,
                               atol=1e-9)


def test_alg1_endpoint_closed_form():
    """One stage, V_T = 0, non-recombining end points: with lam > 0 the best
    action discharges the largest feasible power of p_hat; with lam < 0 it
    charges the largest feasible |p| (eq. 4 restricted to the grid)."""
    eta, delta, p_max, s_max = math.sqrt(0.85), 0.1, 1.0, 4.0
    p_hat, n_c, n_d = O.paper_action_grid(p_max, delta, eta)
    S = 41
    for lam in (37.0, -12.0):
        V = O.paper_alg1(s_max, delta, p_max, eta, np.array([[lam]]), np.array([[1.0]]))
        for i in range(S):
            s = i * delta
            if lam > 0:
                if s >= p_max / eta - 1e-12:
                    p = p_max
                else:
                    p = min(int(math.floor(s / delta + 1e-9)), n_d - 1) * delta * eta
            else:
                if s + p_max * eta <= s_max + 1e-12:
                    p = -p_max
                else:
                    p = -min(int(math.floor((s_max - s) / delta + 1e-9)), n_c - 1) * delta / eta
            assert V[0, i] == pytest.approx(lam * p, rel=1e-12, abs=1e-12), (lam, i)


def test_alg1_interpolation_two_stages():
    """Two stages with end points off the grid: the stage-1 value of the
    end-point actions is the linear interpolation (np.interp) of V_hat_1
    between grid points (Alg. 1, next-stage value step)."""
    eta, delta, p_max, s_max = math.sqrt(0.85), 0.1, 0.35, 2.0
    lam = np.array([[20.0, 55.0], [61.0, 8.0]])
    pi = np.array([[0.3, 0.7], [0.6, 0.4]])
    V = O.paper_alg1(s_max, delta, p_max, eta, lam, pi)
    p_hat, _, _ = O.paper_action_grid(p_max, delta, eta)
    F = O.paper_F(p_hat, eta)
    S = int(round(s_max / delta)) + 1
    grid = np.arange(S) * delta
    V1 = V[1]
    ref = np.zeros(S)
    for i in range(S):
        q = []
        for r in range(2):
            best = -math.inf
            for p, f in zip(p_hat, F):
                x = grid[i] + f
                if x < -1e-12 or x > s_max + 1e-12:
                    continue
                best = max(best, lam[0, r] * p + np.interp(min(max(x, 0), s_max), grid, V1))
            q.append(best)
        ref[i] = pi[0] @ np.array(q)
    np.testing.assert_allclose(V[0], ref, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------- LP upper bound

def _lp_value(price, s_max, x_dis, x_chg, eta_c, eta_d, c_dis, s0):
    """Deterministic arbitrage LP (eq. 1 with the p^c/p^d split of eq. 3a-3b,
    complementarity dropped): per stage variables p^d, p^c >= 0 (grid MWh) and
    the SoC s_t; s_t = s_{t-1} + eta_c p^c - p^d/eta_d, 0 <= s_t <= s_max,
    stored-energy limits p^d/eta_d <= x_dis, eta_c p^c <= x_chg.  Objective
    sum lam_t (p^d - p^c) - c_dis p^d / eta_d."""
    from scipy.optimize import linprog
    T = len(price)
    nv = 3 * T  # [pd_t, pc_t, s_t]
    c = np.zeros(nv)
    for t in range(T):
        c[t] = -(price[t] - c_dis / eta_d)
        c[T + t] = price[t]
    Aeq = np.zeros((T, nv))
    beq = np.zeros(T)
    for t in range(T):
        Aeq[t, 2 * T + t] = 1.0
        if t > 0:
            Aeq[t, 2 * T + t - 1] = -1.0
        else:
            beq[t] = s0
        Aeq[t, t] = 1.0 / eta_d
        Aeq[t, T + t] = -eta_c
    bounds = ([(0, x_dis * eta_d)] * T + [(0, x_chg / eta_c)] * T + [(0, s_max)] * T)
    res = linprog(c, A_eq=Aeq, b_eq=beq, bounds=bounds, method="highs")
    assert res.status == 0
    return -res.fun


def test_dp_below_lp_and_gap_shrinks():
    """Sec. V-A: the discretised DP is a restriction of the continuous
    problem, so its value is below the LP; the gap shrinks as delta -> 0."""
    rng = np.random.default_rng(5)
    T = 48
    price = (40 + 25 * np.sin(np.arange(T) / 3.0) + rng.normal(0, 8, T)).astype(np.float32)
    s_max, eta_c, eta_d = 2.0, 0.9, 0.93
    x_lim = 0.3   # MWh of stored energy per stage; not a divisor of s_max
    c_per = 2.0   # $ per MWh of stored energy discharged
    lp = _lp_value(price.astype(np.float64), s_max, x_lim, x_lim, eta_c, eta_d, c_per, 0.0)
    gaps = []
    for N in (11, 21, 41, 81, 161):
        delta = s_max / (N - 1)
        D = int(math.floor(x_lim / delta + 1e-9))   # the DP may not exceed the limit
        inst = I.random_instance(0, T, N, 1, D, D, 1, eta=(eta_c, eta_d), s_max=s_max,
                                 cost="zero", terminal="zero")
        inst.price[:] = price[:, None]
        sh = np.arange(inst.A) - D
        inst.cost = np.where(sh < 0, c_per * (-sh) * delta, 0.0).astype(np.float32)
        inst.s0 = 0
        dp = O.objective(inst, O.solve(inst)["V1"])
        assert dp <= lp + 1e-6
        gaps.append((lp - dp) / abs(lp))
    assert gaps[-1] < gaps[0]
    assert gaps[-1] < 0.01


# --------------------------------------------------------------- invariants

def test_base_case_and_nonnegativity():
    inst = I.random_instance(31, 10, 30, 4, 5, 3, 1, neg_prob=0.3, terminal="zero", cost="linear")
    r = O.solve(inst, keep_V=True)
    assert np.all(r["V"][-1] == 0.0)             # V_{T+1} = 0 (eq. 6 base case)
    assert np.all(r["V"] >= -1e-12)              # idling is free and feasible


def test_concavity_in_soc():
    """Nonnegative prices, convex cost in the action, concave terminal and
    eta_c eta_d <= 1 keep V_t concave in SoC for every price state."""
    inst = I.random_instance(32, 12, 60, 5, 6, 4, 1, neg_prob=0.0, terminal="linear", cost="linear")
    r = O.solve(inst, keep_V=True)
    second = r["V"][:, 0, 2:, :] - 2 * r["V"][:, 0, 1:-1, :] + r["V"][:, 0, :-2, :]
    assert second.max() <= 1e-9 * np.abs(r["V"]).max()


def test_tie_rule_smallest_action():
    """All payoffs and values zero: every feasible action ties, the policy is
    the smallest feasible action index (deepest feasible discharge)."""
    inst = I.random_instance(33, 3, 9, 2, 3, 2, 1, cost="zero", terminal="zero")
    inst.price[:] = 0
    r = O.solve(inst)
    for s in range(inst.N):
        assert np.all(r["policy"][:, 0, s, :] == max(0, inst.D_dis - s))
        assert np.all(r["gap"][:, 0, s, :] == 0.0)


@pytest.mark.parametrize("modes", [1, 2])
def test_action_value_reproduces_bellman_step(modes):
    """action_value (the value of one given action) against the C oracle's
    Bellman step on the same EV: at the oracle's policy it equals V_t bit for
    bit, no action exceeds V_t, the best other action sits exactly `gap`
    below, and infeasible shifts are -inf (a dropped payoff term, a wrong
    sign of the switch cost or a wrong next mode breaks one of these)."""
    inst = I.random_instance(36 + modes, 5, 23, 3, 4, 6, modes, neg_prob=0.3, cost="nonconvex",
                             switch_cost=2.5, eta=(0.87, 0.93))
    r = O.solve(inst, keep_V=True, keep_EV=True)
    M, N, K, A = inst.n_modes, inst.N, inst.K, inst.A
    m, s, k, a = np.meshgrid(np.arange(M), np.arange(N), np.arange(K), np.arange(A),
                             indexing="ij")
    for t in range(1, inst.T + 1):
        q = O.action_value(inst, t, r["EV"][t - 1], m, s, k, a)
        V = r["V"][t - 1]
        pol = r["policy"][t - 1]
        best = np.take_along_axis(q, pol[..., None], axis=3)[..., 0]
        np.testing.assert_array_equal(best, V)
        assert np.all(q <= V[..., None])
        np.testing.assert_array_equal(q.max(axis=3), V)
        others = q.copy()
        np.put_along_axis(others, pol[..., None], -np.inf, axis=3)
        second = others.max(axis=3)
        fin = np.isfinite(second)
        np.testing.assert_array_equal((V - second)[fin], r["gap"][t - 1][fin])
        shift = s + (a - inst.D_dis)
        assert np.all(np.isneginf(q[(shift < 0) | (shift > N - 1)]))


# ------------------------------------------------------------- Monte Carlo

@pytest.mark.parametrize("which", ["config1", "modes"])
def test_monte_carlo_reproduces_J(which):
    if which == "config1":
        inst = I.config1()
    else:
        inst = I.random_instance(41, 20, 40, 4, 5, 5, 2, neg_prob=0.2, switch_cost=12.0)
        inst.s0 = 20
    r = O.solve(inst)
    J = O.objective(inst, r["V1"])
    mean, se = O.mc_simulate(inst, r["policy"], 1_000_000, seed=3)
    assert abs(mean - J) <= 3 * se, (mean, J, se)


# ------------------------------------------------ occupancy and gradients

def _tie_free(seed=51, modes=1):
    inst = I.random_instance(seed, 6, 25, 3, 3, 3, modes, neg_prob=0.2, switch_cost=5.0,
                             cost="linear")
    inst.s0 = 12
    return inst


@pytest.mark.parametrize("modes", [1, 2])
def test_occupancy_identity(modes):
    inst = _tie_free(52, modes)
    r = O.solve(inst, keep_V=True)
    occ = O.occupancy(inst, r["policy"], r["V"])
    assert occ["J"] == pytest.approx(O.objective(inst, r["V1"]), rel=1e-14)
    assert occ["J_occ"] == pytest.approx(occ["J"], rel=1e-12)
    # probability mass is conserved up to the float32 row-sum error of trans
    rowdev = np.abs(inst.trans.astype(np.float64).sum(axis=2) - 1.0).max()
    np.testing.assert_allclose(occ["mass"], 1.0, atol=(inst.T + 1) * (rowdev + 1e-7))


def _J(inst, **kw):
    return O.objective(inst, O.solve(inst, keep_policy=False, **kw)["V1"])


def _min_gap(inst):
    r = O.solve(inst, keep_V=True)
    occ = O.occupancy(inst, r["policy"], r["V"])
    return r, occ


@pytest.mark.parametrize("modes", [1, 2])
def test_gradients_vs_central_differences(modes):
    inst = _tie_free(53, modes)
    r, occ = _min_gap(inst)
    price = inst.price.astype(np.float64)
    trans = inst.trans.astype(np.float64)
    h = 1e-3
    for (t, k) in [(0, 0), (2, 1), (5, 2), (3, 0)]:
        p1 = price.copy(); p1[t, k] += h
        p2 = price.copy(); p2[t, k] -= h
        fd = (_J(inst, price=p1) - _J(inst, price=p2)) / (2 * h)
        assert fd == pytest.approx(occ["d_price"][t, k], rel=1e-6, abs=1e-8)
    hp = 1e-6
    for (t, k, k2) in [(0, 0, 1), (2, 1, 2), (4, 2, 0)]:
        q1 = trans.copy(); q1[t, k, k2] += hp
        q2 = trans.copy(); q2[t, k, k2] -= hp
        fd = (_J(inst, trans=q1) - _J(inst, trans=q2)) / (2 * hp)
        assert fd == pytest.approx(occ["d_trans"][t, k, k2], rel=1e-5, abs=1e-6)
    he = 1e-5
    fd = (_J(inst, eta_c=inst.eta_c + he) - _J(inst, eta_c=inst.eta_c - he)) / (2 * he)
    assert fd == pytest.approx(occ["d_eta_c"], rel=1e-5, abs=1e-6)
    fd = (_J(inst, eta_d=inst.eta_d + he) - _J(inst, eta_d=inst.eta_d - he)) / (2 * he)
    assert fd == pytest.approx(occ["d_eta_d"], rel=1e-5, abs=1e-6)


@pytest.mark.parametrize("modes", [1, 2])
def test_input_gradients_vs_central_differences(modes):
    """Per-action cost, switch cost, terminal value and initial price-state
    distribution: central differences of the FP64 DP against the occupancy
    pass (a planted sign error or a dropped term fails these)."""
    inst = _tie_free(55, modes)
    r, occ = _min_gap(inst)
    cost = inst.cost.astype(np.float64)
    h = 1e-4
    chosen = np.unique(r["policy"])
    unused = [a for a in range(inst.A) if a not in set(chosen.tolist())]
    for a in list(chosen[:3]) + unused[:1]:
        c1 = cost.copy(); c1[a] += h
        c2 = cost.copy(); c2[a] -= h
        fd = (_J(inst, cost=c1) - _J(inst, cost=c2)) / (2 * h)
        assert fd == pytest.approx(occ["d_cost"][a], rel=1e-6, abs=1e-9)
    assert any(occ["d_cost"][a] < 0 for a in chosen) and all(occ["d_cost"][a] == 0 for a in unused)
    # the cost gradient counts every decision once: total occupancy mass
    assert -occ["d_cost"].sum() == pytest.approx(occ["mass"].sum(), rel=1e-12)
    if modes == 2:
        hs = 1e-4
        fd = (_J(inst, switch_cost=inst.switch_cost + hs)
              - _J(inst, switch_cost=inst.switch_cost - hs)) / (2 * hs)
        assert fd == pytest.approx(occ["d_switch"], rel=1e-6, abs=1e-9)
    term = inst.terminal.astype(np.float64)
    flat = np.argsort(-occ["d_terminal"].ravel())[:3]
    for i in list(flat) + [int(np.argmin(occ["d_terminal"].ravel()))]:
        idx = np.unravel_index(i, term.shape)
        t1 = term.copy(); t1[idx] += h
        t2 = term.copy(); t2[idx] -= h
        fd = (_J(inst, terminal=t1) - _J(inst, terminal=t2)) / (2 * h)
        assert fd == pytest.approx(occ["d_terminal"][idx], rel=1e-6, abs=1e-9)
    # the final occupancy is a distribution (up to the float32 row sums of P)
    rowdev = np.abs(inst.trans.astype(np.float64).sum(axis=2) - 1.0).max()
    assert occ["d_terminal"].sum() == pytest.approx(1.0, abs=(inst.T + 1) * (rowdev + 1e-7))
    # J is linear in mu0
    import copy
    for k in range(inst.K):
        i1 = copy.copy(inst); i1.mu0 = inst.mu0.astype(np.float64).copy(); i1.mu0[k] += 0.5
        assert O.objective(i1, r["V1"]) - O.objective(inst, r["V1"]) == pytest.approx(
            0.5 * occ["d_mu0"][k], rel=1e-12, abs=1e-12)


# --------------------------------------------------------------------- hull

def _hull_brute(y):
    """Strict vertices of the upper envelope by definition: an interior
    point is a vertex iff it lies strictly above every chord between a point
    on its left and a point on its right (exact rational arithmetic)."""
    n = len(y)
    Y = [Fraction(float(v)) for v in y]
    out = [0]
    for i in range(1, n - 1):
        ok = True
        for j in range(i):
            for l in range(i + 1, n):
                chord = Y[j] + (Y[l] - Y[j]) * Fraction(i - j, l - j)
                if Y[i] <= chord:
                    ok = False
                    break
            if not ok:
                break
        if ok:
            out.append(i)
    if n > 1:
        out.append(n - 1)
    return np.array(out)


@pytest.mark.parametrize("seed", range(8))
def test_hull_bruteforce(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 64))
    kind = seed % 4
    if kind == 0:
        y = rng.normal(size=n)
    elif kind == 1:   # concave with collinear runs
        y = -np.abs(np.arange(n) - n / 3).astype(np.float64) * 2.0
    elif kind == 2:   # integer-valued, many exact collinearities and ties
        y = rng.integers(-3, 4, size=n).astype(np.float64)
    else:             # float32 values of a concave-ish value function
        y = (np.sqrt(np.arange(n) + 1.0) * 10 + rng.normal(0, 0.05, n)).astype(np.float32)
    y = np.asarray(y, dtype=np.float32).astype(np.float64)
    h = O.hull(y)
    np.testing.assert_array_equal(h, _hull_brute(y))
    # the envelope value at each grid point equals the best chord through it
    env = np.interp(np.arange(n), h, y[h])
    for i in range(n):
        best = y[i]
        for j in range(i + 1):
            for l in range(i, n):
                if l > j:
                    best = max(best, y[j] + (y[l] - y[j]) * (i - j) / (l - j))
        assert env[i] == pytest.approx(best, rel=1e-12, abs=1e-12)
    s = O.hull_slopes(y, h, 1.0)
    assert np.all(np.diff(s) < 0)        # monotone bid prices (eq. 11)



# ----------------------------------------------- bid curves and clearing (Sec. II-C, V)

def test_paper_bids_envelope_by_brute_force():
    """The bid vertices are exactly the points above every chord (the
    envelope definition) and the prices are monotone non-decreasing."""
    rng = np.random.default_rng(11)
    S, s_max, p_max, eta, tau = 41, 4.0, 1.0, math.sqrt(0.85), 1.0
    for trial in range(6):
        v = np.cumsum(rng.normal(2.0, 3.0, size=S)).astype(np.float32)  # non-concave
        s = int(rng.integers(0, S))
        idx, prices = O.paper_bids(S, s_max, p_max, eta, tau, v, s)
        p, f = O._shifts(S, s_max, p_max, eta, tau)
        pts = [(a, p[a], O._v_at(v, s + f[a])) for a in range(len(p))
               if -1e-9 <= s + f[a] <= S - 1 + 1e-9]
        xs = [Fraction(x) for _, x, _ in pts]
        ys = [Fraction(y) for _, _, y in pts]
        brute = [pts[0][0]]
        for i in range(1, len(pts) - 1):
            if all(ys[i] > ys[j] + (ys[l] - ys[j]) * (xs[i] - xs[j]) / (xs[l] - xs[j])
                   for j in range(i) for l in range(i + 1, len(pts))):
                brute.append(pts[i][0])
        brute.append(pts[-1][0])
        assert idx == brute
        assert all(b >= a for a, b in zip(prices, prices[1:]))


def test_paper_bids_concave_value_keeps_every_action():
    """V concave and increasing in SoC (Sec. II-C): U(p; s) is concave in p,
    every feasible action is on the envelope (up to collinear runs) and the
    bid at zero power lies between the discharge and charge marginal values."""
    S, s_max, p_max, eta, tau = 81, 4.0, 1.0, math.sqrt(0.85), 1.0
    x = np.arange(S) * (s_max / (S - 1))
    v = (50.0 * x - 4.0 * x ** 2).astype(np.float32)
    idx, prices = O.paper_bids(S, s_max, p_max, eta, tau, v, 40)
    p, f = O._shifts(S, s_max, p_max, eta, tau)
    feas = [a for a in range(len(p)) if -1e-9 <= 40 + f[a] <= S - 1 + 1e-9]
    assert len(idx) >= len(feas) - 2
    assert all(b >= a for a, b in zip(prices, prices[1:]))


def test_paper_clear_reproduces_dp_value_in_expectation():
    """Paths drawn from the model's own price samples: the clearing policy
    is the DP's maximiser, so the mean revenue is V_0(s0) (zero terminal,
    eta = 1 so that every action stays on the grid) within 3 standard errors."""
    prob = I.iid_problem(21, 8, 21, 5, 2.0, eta=1.0)
    V = O.paper_alg1(prob.s_max, prob.delta, prob.p_max, prob.eta, prob.lam_hat, prob.pi_hat)
    rng = np.random.default_rng(3)
    n = 4000
    s0 = 1.0
    revs = []
    for _ in range(n):
        k = [rng.choice(prob.R, p=prob.pi_hat[t].astype(np.float64) / prob.pi_hat[t].sum())
             for t in range(prob.T)]
        lam = prob.lam_hat[np.arange(prob.T), k]
        revs.append(O.paper_clear(prob.S, prob.s_max, prob.p_max, prob.eta, prob.tau, V, lam, s0)[0])
    revs = np.array(revs)
    se = revs.std(ddof=1) / math.sqrt(n)
    target = V[0][int(round(s0 / prob.delta))]
    assert abs(revs.mean() - target) <= 3 * se + 1e-9, (revs.mean(), target, se)


# ------------------------------------ Markov bids at a SoC state (eq. 8-11)

def _bid_inst(N, D_dis, D_chg, eta_c, eta_d, s_max=4.0, tau=0.25):
    inst = I.random_instance(0, 2, N, 2, D_dis, D_chg, 1)
    inst.eta_c, inst.eta_d, inst.s_max, inst.tau = eta_c, eta_d, s_max, tau
    return inst


def test_markov_bids_linear_value_closed_form():
    """EV linear in SoC with marginal value g per MWh of stored energy, s
    inside the window: buying grid energy adds g eta_c per MWh, selling needs
    g / eta_d per MWh.  For g > 0 the two sides are monotone (g eta_c <
    g / eta_d) and s stays a vertex; for g < 0 they cross and the re-hull over
    power merges them into one segment at the average
    g (hi - lo) / ((s - lo) eta_d + (hi - s) / eta_c)."""
    N, Dd, Dc, ec, ed = 61, 7, 11, 0.9, 0.8
    inst = _bid_inst(N, Dd, Dc, ec, ed)
    delta = inst.s_max / (N - 1)
    s, lo, hi = 30, 30 - Dd, 30 + Dc
    for g in (37.0, -12.0):
        y = g * delta * np.arange(N)
        xs, ps, prices = O.markov_bids_at(inst, y, s)
        if g > 0:
            assert xs == [hi, s, lo]
            assert prices == pytest.approx([g * ec, g / ed], rel=1e-12)
            assert ps == pytest.approx([-(hi - s) * delta / (ec * inst.tau), 0.0,
                                        (s - lo) * delta * ed / inst.tau], rel=1e-12)
        else:
            assert xs == [hi, lo]
            assert prices == pytest.approx([g * (hi - lo) / ((s - lo) * ed + (hi - s) / ec)],
                                           rel=1e-12)


def test_markov_bids_unit_efficiency_are_soc_slopes():
    """eta_c = eta_d = 1: power is linear in SoC on both sides, so the bid
    vertices are the window's ends and the SoC-envelope vertices inside it,
    and every price is the envelope slope of its SoC segment."""
    rng = np.random.default_rng(4)
    N = 80
    inst = _bid_inst(N, 12, 9, 1.0, 1.0)
    delta = inst.s_max / (N - 1)
    for trial in range(6):
        y = np.cumsum(rng.normal(1.0, 4.0, size=N)).astype(np.float32).astype(np.float64)
        s = int(rng.integers(0, N))
        lo, hi = max(0, s - 12), min(N - 1, s + 9)
        h = O.hull(y)
        xs, _, prices = O.markov_bids_at(inst, y, s)
        expect = sorted({lo, hi} | {int(v) for v in h if lo < v < hi}, reverse=True)
        env = np.interp(np.arange(N), h, y[h])
        want = [(env[a] - env[b]) / ((a - b) * delta) for a, b in zip(xs, xs[1:])]
        assert prices == pytest.approx(want, rel=1e-9, abs=1e-9)
        if xs != expect:
            # s on an envelope segment is collinear in exact arithmetic; its
            # interpolated value may round above the chord, which leaves it as
            # a vertex between two equal prices
            q = xs.index(s)
            assert s not in expect and [x for x in xs if x != s] == expect
            assert prices[q - 1] == pytest.approx(prices[q], rel=1e-9, abs=1e-9)


def test_markov_bids_envelope_and_merit_order_by_brute_force():
    """Vertices are exactly the candidate points above every chord (exact
    rationals), prices never fall, and at any price lam the curve clears the
    power that maximises lam p tau + E(s + shift(p)) over every grid point of
    the window (E the SoC envelope, taken by linear interpolation of the
    envelope vertices)."""
    rng = np.random.default_rng(12)
    N = 70
    for trial in range(8):
        Dd, Dc = int(rng.integers(0, 20)), int(rng.integers(0, 20))
        ec, ed = float(rng.uniform(0.8, 1.0)), float(rng.uniform(0.8, 1.0))
        inst = _bid_inst(N, Dd, Dc, ec, ed, tau=float(rng.choice([1.0, 0.25])))
        delta = inst.s_max / (N - 1)
        y = np.cumsum(rng.normal(0.5, 3.0, size=N)).astype(np.float32).astype(np.float64)
        s = int(rng.integers(0, N))
        lo, hi = max(0, s - Dd), min(N - 1, s + Dc)
        xs, ps, prices = O.markov_bids_at(inst, y, s)
        assert all(b >= a for a, b in zip(prices, prices[1:]))
        h = O.hull(y)
        env = np.interp(np.arange(N), h, y[h])

        def power(x):
            e = (s - x) * delta
            return (e * ed if x <= s else e / ec) / inst.tau
        # candidate points in ascending power, exact-rational envelope test
        cand = sorted({lo, hi, s} | {int(v) for v in h if lo < v < hi}, reverse=True)
        P = [Fraction(power(x)) for x in cand]
        U = [Fraction(float(O.envelope_at(y, h, x))) for x in cand]
        brute = [cand[0]] + [cand[i] for i in range(1, len(cand) - 1)
                             if all(U[i] > U[j] + (U[l] - U[j]) * (P[i] - P[j]) / (P[l] - P[j])
                                    for j in range(i) for l in range(i + 1, len(cand)))]
        if len(cand) > 1:
            brute.append(cand[-1])
        assert xs == brute
        # merit order
        window = range(lo, hi + 1)
        for lam in rng.uniform(-80.0, 80.0, size=25):
            best = max(lam * power(x) * inst.tau + env[x] for x in window)
            q = sum(1 for pr in prices if pr < lam)
            got = lam * ps[q] * inst.tau + O.envelope_at(y, h, xs[q])
            assert got == pytest.approx(best, rel=1e-10, abs=1e-9)
