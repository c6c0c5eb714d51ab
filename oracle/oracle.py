"""FP64 oracle for the storage-arbitrage DP: Python side.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the benchmark's CPU-baseline leg; never by the product path.  It
shares no code with the CUDA library.

Pieces:
  * ``solve``      -- ctypes wrapper of the C backward induction (eq. 4-6 with
                      a Markov price chain, Alg. 1 in plain loops);
  * ``action_value`` -- the FP64 value of one given action in one state
                      (payoff + EV at the shifted SoC, eq. 5), to check that
                      a decision taken elsewhere is a maximiser;
  * ``hull``       -- monotone-chain upper envelope (eq. 10-11);
  * ``markov_bids_at`` -- price-quantity bids at one SoC state from that
                      envelope, re-convexified over grid power (eq. 8-11);
  * ``occupancy``  -- forward state-occupancy pass and the envelope-theorem
                      gradients of J;
  * ``paper_alg1`` -- Algorithm 1 taken literally with numpy: the eq. 13 action
                      grid with its two interpolated end points, the
                      stagewise-independent price samples of eq. 14;
  * ``mc_simulate``-- Monte Carlo forward simulation of a stored policy.

Readings of the paper taken here (garbled or silent passages):
  * the next-state proxy of Alg. 1 projects sigma onto [0, s_max], i.e.
    max{0, min{sigma, s_max}} (the printed min/max order is swapped);
  * the infeasibility mask uses sigma > s_max (printed as sigma > S);
  * the last entry of F(p_hat) is -p_max/eta (printed without the sign);
  * the interpolation factor is 0 where z+ == z- (printed as 0/0);
  * the stage loop produces V_{T-1}..V_0 from stages T..1 (a t = 0 iteration
    would need lambda_0, which does not exist).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "esdp_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, no FP contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("N", ctypes.c_int32), ("K", ctypes.c_int32),
                ("A", ctypes.c_int32), ("D_dis", ctypes.c_int32), ("D_chg", ctypes.c_int32),
                ("n_modes", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("s_max", ctypes.c_double), ("eta_c", ctypes.c_double),
                ("eta_d", ctypes.c_double), ("switch_cost", ctypes.c_double)]


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        _lib.orc_solve.argtypes = [ctypes.POINTER(_Problem), dp, dp, dp, dp, dp, dp, ip, dp, dp,
                                   ctypes.c_int]
        _lib.orc_hull.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip]
        _lib.orc_occupancy.argtypes = [ctypes.POINTER(_Problem), dp, dp, dp, ip, dp, ctypes.c_int,
                                       dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
    return _lib


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _problem(inst, **over) -> _Problem:
    d = dict(T=inst.T, N=inst.N, K=inst.K, A=inst.A, D_dis=inst.D_dis, D_chg=inst.D_chg,
             n_modes=inst.n_modes, s_max=inst.s_max, eta_c=inst.eta_c, eta_d=inst.eta_d,
             switch_cost=inst.switch_cost)
    d.update(over)
    return _Problem(T=d["T"], N=d["N"], K=d["K"], A=d["A"], D_dis=d["D_dis"], D_chg=d["D_chg"],
                    n_modes=d["n_modes"], pad_=0, s_max=d["s_max"], eta_c=d["eta_c"],
                    eta_d=d["eta_d"], switch_cost=d["switch_cost"])


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def solve(inst, *, keep_V: bool = False, keep_EV: bool = False, keep_policy: bool = True,
          nthreads: int = 1, price=None, trans=None, cost=None, terminal=None, **over) -> dict:
    """Backward induction in FP64.  Returns V1 [M,N,K] and, on request,
    V [T+1,M,N,K] (V_t at index t-1, V_{T+1} last), EV [T,M,N,K],
    policy/gap [T,M,N,K].  Array overrides allow finite differences."""
    lib = _load()
    p = _problem(inst, **over)
    T, M, N, K = p.T, p.n_modes, p.N, p.K
    price = _f64(inst.price if price is None else price)
    trans = _f64(inst.trans if trans is None else trans)
    cost = _f64(inst.cost if cost is None else cost)
    terminal = _f64(inst.terminal if terminal is None else terminal)
    assert price.shape == (T, K) and trans.shape == (T, K, K)
    out = {"V1": np.empty((M, N, K))}
    out["V"] = np.empty((T + 1, M, N, K)) if keep_V else None
    out["EV"] = np.empty((T, M, N, K)) if keep_EV else None
    out["policy"] = np.empty((T, M, N, K), np.int32) if keep_policy else None
    out["gap"] = np.empty((T, M, N, K)) if keep_policy else None
    rc = lib.orc_solve(ctypes.byref(p), _dp(price), _dp(trans), _dp(cost), _dp(terminal),
                       _dp(out["V"]), _dp(out["EV"]), _ip(out["policy"]), _dp(out["gap"]),
                       _dp(out["V1"]), int(nthreads))
    if rc != 0:
        raise ValueError(f"orc_solve failed ({rc})")
    return out


def action_value(inst, t: int, EV_t: np.ndarray, m, s, k, a, price=None) -> np.ndarray:
    """FP64 value of taking action a in state (m, s, k) at stage t (eq. 5):
    the payoff price[t,k] e_a - cost[a] (- switch cost when a discharge
    leaves mode 1) plus EV_t[m'][s + d][k] at the shifted SoC, d = a - D_dis,
    m' the mode after the action; -inf where s + d leaves the grid (eq. 4).
    EV_t: [M, N, K] (any float dtype, promoted to float64); m, s, k, a:
    integer arrays of one shape (broadcast).  The same double operations, in
    the same order, as the C oracle's Bellman step, so that at the oracle's
    own policy it reproduces V_t bit for bit."""
    m, s, k, a = (np.asarray(x, dtype=np.int64) for x in np.broadcast_arrays(m, s, k, a))
    d = a - inst.D_dis
    delta = inst.s_max / float(inst.N - 1)
    e = np.where(d < 0, (-d.astype(np.float64) * delta) * inst.eta_d,
                 np.where(d > 0, (-d.astype(np.float64) * delta) / inst.eta_c, 0.0))
    lam = np.asarray(inst.price if price is None else price, np.float64)[t - 1, k]
    r = lam * e - np.asarray(inst.cost, np.float64)[a]
    if inst.n_modes == 2:
        r = np.where((m == 1) & (d < 0), r - inst.switch_cost, r)
        m2 = np.where(d < 0, 0, np.where(d > 0, 1, m))
    else:
        m2 = np.zeros_like(m)
    s2 = s + d
    ok = (s2 >= 0) & (s2 <= inst.N - 1)
    ev = np.asarray(EV_t, np.float64)[m2, np.clip(s2, 0, inst.N - 1), k]
    return np.where(ok, r + ev, -np.inf)


def objective(inst, V1: np.ndarray) -> float:
    """J = sum_k mu0[k] V_1[mode 0][s0][k]."""
    return float(np.dot(inst.mu0.astype(np.float64), V1[0, inst.s0, :]))


def hull(y: np.ndarray) -> np.ndarray:
    """Vertex indices of the upper concave envelope of (i, y[i])."""
    lib = _load()
    y = _f64(y)
    idx = np.empty(len(y), np.int32)
    n = lib.orc_hull(len(y), _dp(y), 1, _ip(idx))
    return idx[:n].copy()


def hull_slopes(y: np.ndarray, idx: np.ndarray, delta: float) -> np.ndarray:
    """Slopes of the envelope between consecutive vertices, per MWh."""
    y = _f64(y)
    return (y[idx[1:]] - y[idx[:-1]]) / ((idx[1:] - idx[:-1]) * delta)


def bid_curves(inst, EV: np.ndarray):
    """Envelope of EV_t[m, :, k] over SoC for every (t, m, k).

    EV: [T, M, N, K] (any float dtype; promoted exactly to float64).
    Returns (n_bp [T,M,K], idx [T,M,K,N] padded with -1, slope [T,M,K,N-1]
    padded with nan, per MWh)."""
    T, M, N, K = EV.shape
    n_bp = np.zeros((T, M, K), np.int32)
    idx = np.full((T, M, K, N), -1, np.int32)
    slope = np.full((T, M, K, max(N - 1, 1)), np.nan)
    for t in range(T):
        for m in range(M):
            for k in range(K):
                y = np.asarray(EV[t, m, :, k], dtype=np.float64)
                h = hull(y)
                n_bp[t, m, k] = len(h)
                idx[t, m, k, :len(h)] = h
                slope[t, m, k, :len(h) - 1] = hull_slopes(y, h, inst.delta)
    return n_bp, idx, slope


def occupancy(inst, policy: np.ndarray, V: np.ndarray, *, price=None, trans=None, cost=None,
              **over) -> dict:
    """Forward occupancy under `policy` [T,M,N,K] int32 with values `V`
    [T+1,M,N,K]; returns J, J_occ and the gradients."""
    lib = _load()
    p = _problem(inst, **over)
    T, K = p.T, p.K
    price = _f64(inst.price if price is None else price)
    trans = _f64(inst.trans if trans is None else trans)
    cost = _f64(inst.cost if cost is None else cost)
    policy = np.ascontiguousarray(policy.astype(np.int32))
    V = _f64(V)
    mu0 = _f64(inst.mu0)
    J = np.zeros(1)
    J_occ = np.zeros(1)
    dprice = np.zeros((T, K))
    dtrans = np.zeros((T, K, K))
    dc = np.zeros(1)
    dd = np.zeros(1)
    er = np.zeros(T)
    mass = np.zeros(T)
    dcost = np.zeros(p.A)
    dsw = np.zeros(1)
    dterm = np.zeros((p.n_modes, p.N, K))
    rc = lib.orc_occupancy(ctypes.byref(p), _dp(price), _dp(trans), _dp(cost), _ip(policy),
                           _dp(V), int(inst.s0), _dp(mu0), _dp(J), _dp(J_occ), _dp(dprice),
                           _dp(dtrans), _dp(dc), _dp(dd), _dp(er), _dp(mass), _dp(dcost),
                           _dp(dsw), _dp(dterm))
    if rc != 0:
        raise ValueError(f"orc_occupancy failed ({rc})")
    # J = sum_k mu0[k] V_1[0][s0][k] is linear in mu0
    d_mu0 = np.asarray(V[0, 0, inst.s0, :], dtype=np.float64).copy()
    return {"J": float(J[0]), "J_occ": float(J_occ[0]), "d_price": dprice, "d_trans": dtrans,
            "d_eta_c": float(dc[0]), "d_eta_d": float(dd[0]), "exp_reward": er, "mass": mass,
            "d_cost": dcost, "d_switch": float(dsw[0]), "d_terminal": dterm, "d_mu0": d_mu0}


# --------------------------------------------------------------------------
# Algorithm 1, literally (stagewise-independent prices, eq. 13 action grid)
# --------------------------------------------------------------------------

def paper_action_grid(p_max: float, delta: float, eta: float):
    """The discretised power actions of eq. 13 and their count P.

    Charge actions (p < 0) are -j delta/eta for j = 1..n_c-1 plus the end
    point -p_max; discharge actions are j delta eta for j = 1..n_d-1 plus the
    end point p_max; n_c = ceil(p_max eta / delta), n_d = ceil(p_max /
    (delta eta)), P = n_c + n_d + 1."""
    n_c = int(math.ceil(p_max * eta / delta - 1e-12))
    n_d = int(math.ceil(p_max / (delta * eta) - 1e-12))
    chg = [-p_max] + [-(j * delta / eta) for j in range(n_c - 1, 0, -1)]
    dis = [j * delta * eta for j in range(1, n_d)] + [p_max]
    p_hat = np.array(chg + [0.0] + dis)
    assert len(p_hat) == n_c + n_d + 1
    return p_hat, n_c, n_d


def paper_F(p: np.ndarray, eta: float) -> np.ndarray:
    """State transition of eq. 2: -p/eta when discharging, -eta p when charging."""
    return np.where(p >= 0, -p / eta, -eta * p)


def paper_alg1(s_max: float, delta: float, p_max: float, eta: float, lam_hat: np.ndarray,
               pi_hat: np.ndarray, snap: float = 1e-9, *, terminal=None, tau: float = 1.0,
               keep_policy: bool = False):
    """Algorithm 1 in numpy.

    lam_hat, pi_hat: [T, R] price samples and probabilities for stages 1..T.
    Returns V_hat [T+1, S]: V_hat[t] is the expected value vector
    V_hat_t for t = 0..T (V_hat_T = 0, the base case, or `terminal`).
    Stages last `tau` hours (the paper's are hourly: tau = 1): payoff
    lam * p * tau, SoC change F(p) * tau.  With keep_policy also the argmax
    action index (first maximiser) and the top-two gap per [t-1, s, r].

    `snap` absorbs floating-point noise in sigma/delta so that states that
    the paper's recombining grid puts exactly on grid points are treated as
    such (the paper assumes exact arithmetic for these columns)."""
    T, R = lam_hat.shape
    n_s = int(round(s_max / delta))
    S = n_s + 1
    s_hat = np.arange(S) * delta
    p_hat, _, _ = paper_action_grid(p_max, delta, eta)
    P = len(p_hat)
    sigma = s_hat[:, None] + tau * paper_F(p_hat, eta)[None, :]      # next-state levels
    z = np.clip(sigma, 0.0, s_max) / delta + 1.0                       # next-state proxies
    zr = np.round(z)
    z = np.where(np.abs(z - zr) < snap, zr, z)
    zm = np.floor(z).astype(np.int64)                                  # next-state indices
    zp = np.ceil(z).astype(np.int64)
    b = np.where(zp > zm, (z - zm) / np.maximum(zp - zm, 1), 0.0)      # interpolation factors
    infeasible = (sigma < -snap * delta) | (sigma > s_max + snap * delta)
    V = np.zeros((T + 1, S))
    if terminal is not None:
        V[T] = np.asarray(terminal, dtype=np.float64)
    pol = np.empty((T, S, R), np.int32) if keep_policy else None
    gap = np.empty((T, S, R)) if keep_policy else None
    lam64 = np.asarray(lam_hat, dtype=np.float64)
    pi64 = np.asarray(pi_hat, dtype=np.float64)
    for t in range(T, 0, -1):
        Vt = V[t]
        Vnext = (1.0 - b) * Vt[zm - 1] + b * Vt[zp - 1]
        Vnext = np.where(infeasible, -np.inf, Vnext)
        Qall = (tau * p_hat[:, None] * lam64[t - 1][None, :])[None, :, :] + Vnext[:, :, None]
        Q = Qall.max(axis=1)                                           # S x R
        if keep_policy:
            pol[t - 1] = Qall.argmax(axis=1)
            top2 = np.partition(np.where(np.isfinite(Qall), Qall, -1e300), P - 2, axis=1)[:, P - 2, :]
            gap[t - 1] = Q - top2
        V[t - 1] = Q @ pi64[t - 1]
    if keep_policy:
        return V, pol, gap
    return V


# --------------------------------------------------------------------------
# Price-quantity bids at a SoC state from the Markov SoC envelope (eq. 8-11)
# --------------------------------------------------------------------------

def envelope_at(y: np.ndarray, h: np.ndarray, x: int) -> float:
    """Value of the upper concave envelope (vertices h of y) at grid point x:
    y at a vertex, else the chord of the two vertices around x,
    y_a + ((y_b - y_a) (x - a)) / (b - a)."""
    j = int(np.searchsorted(h, x))
    if j < len(h) and h[j] == x:
        return float(y[x])
    a, b = int(h[j - 1]), int(h[j])
    ya, yb = float(y[a]), float(y[b])
    return ya + ((yb - ya) * float(x - a)) / float(b - a)


def markov_bids_at(inst, y: np.ndarray, s: int):
    """Bid curve at SoC index s from EV_t[m][.][k] = y [N] (eq. 8-11 on the
    SoC envelope).  Candidate SoC points: the action window's ends
    lo = max(0, s - D_dis), hi = min(N - 1, s + D_chg), s itself and the
    envelope vertices strictly inside the window; each is mapped to grid
    power (discharge, x <= s: p = (((s - x) delta) eta_d) / tau; charge,
    x > s: p = (((s - x) delta) / eta_c) / tau) with U = envelope value.
    Over ascending p the upper concave envelope of (p, U) is taken by the
    monotone chain (a middle point is dropped when
    (U_j - U_i)(p_l - p_i) - (U_l - U_i)(p_j - p_i) <= 0), and segment q sells
    at -(U_{q+1} - U_q) / ((p_{q+1} - p_q) tau).  Returns (SoC indices of the
    vertices, their powers in MW, the segment prices)."""
    y = np.asarray(y, dtype=np.float64)
    N = len(y)
    h = hull(y)
    delta = inst.s_max / (N - 1)
    lo, hi = max(0, s - inst.D_dis), min(N - 1, s + inst.D_chg)
    xs = sorted({lo, hi, s} | {int(v) for v in h if lo < v < hi}, reverse=True)
    pts = []
    for x in xs:  # descending SoC = ascending power
        if x <= s:
            p = (((s - x) * delta) * inst.eta_d) / inst.tau
        else:
            p = (((s - x) * delta) / inst.eta_c) / inst.tau
        pts.append((x, p, envelope_at(y, h, x)))
    chain = []
    for x, p, u in pts:
        while len(chain) >= 2:
            (_, pi, ui), (_, pj, uj) = chain[-2], chain[-1]
            if (uj - ui) * (p - pi) - (u - ui) * (pj - pi) > 0.0:
                break
            chain.pop()
        chain.append((x, p, u))
    prices = [-(chain[q + 1][2] - chain[q][2]) / ((chain[q + 1][1] - chain[q][1]) * inst.tau)
              for q in range(len(chain) - 1)]
    return [c[0] for c in chain], [c[1] for c in chain], prices


# --------------------------------------------------------------------------
# Bid curves (eq. 8-11) and merit-order clearing on Algorithm 1's values
# --------------------------------------------------------------------------

def _v_at(v: np.ndarray, z: float) -> float:
    """V at SoC position z (grid steps): the grid value within 1e-9 of a grid
    point, else linear interpolation (1 - b) V[j] + b V[j+1]."""
    S = len(v)
    j = math.floor(z)
    b = z - j
    if b < 1e-9:
        return float(np.float64(v[max(0, min(S - 1, j))]))
    if b > 1.0 - 1e-9:
        return float(np.float64(v[max(0, min(S - 1, j + 1))]))
    return (1.0 - b) * float(v[j]) + b * float(v[j + 1])


def _shifts(S: int, s_max: float, p_max: float, eta: float, tau: float):
    delta = s_max / (S - 1)
    p_hat, _, _ = paper_action_grid(p_max, delta, eta)
    f = [float(x) * tau / delta for x in paper_F(p_hat, eta)]
    return [float(x) for x in p_hat], f


def paper_bids(S: int, s_max: float, p_max: float, eta: float, tau: float, v: np.ndarray, s: int):
    """Convexified bid curve at grid SoC s from the next-stage values v [S]
    (eq. 8-11): points (p_a, U(p_a; s) = V(s + F(p_a) tau)) of the feasible
    actions, upper concave envelope by the monotone chain over ascending p (a
    middle point is dropped when (y_j - y_i)(x_l - x_i) - (y_l - y_i)(x_j - x_i)
    <= 0), bid prices -(dU/dp)/tau per envelope segment.  Returns (vertex
    action indices, prices)."""
    p, f = _shifts(S, s_max, p_max, eta, tau)
    pts = []
    for a in range(len(p)):
        z = s + f[a]
        if -1e-9 <= z <= S - 1 + 1e-9:
            pts.append((a, p[a], _v_at(v, z)))
    hull = []
    for a, x, y in pts:
        while len(hull) >= 2:
            (_, xi, yi), (_, xj, yj) = hull[-2], hull[-1]
            if (yj - yi) * (x - xi) - (y - yi) * (xj - xi) > 0.0:
                break
            hull.pop()
        hull.append((a, x, y))
    idx = [h[0] for h in hull]
    prices = [-(hull[q + 1][2] - hull[q][2]) / ((hull[q + 1][1] - hull[q][1]) * tau)
              for q in range(len(hull) - 1)]
    return idx, prices


def paper_clear(S: int, s_max: float, p_max: float, eta: float, tau: float, V_all: np.ndarray,
                lam_real: np.ndarray, s0: float):
    """Merit-order clearing of a price-taking storage (Sec. V): at stage t the
    cleared action maximises lam_t p tau + V_t(s + F(p) tau) (the vertex of
    the convexified bid curve crossed by lam_t; the first on ties), the SoC
    moves, lam_t p tau accrues.  Returns (revenue, final SoC in grid steps,
    actions)."""
    p, f = _shifts(S, s_max, p_max, eta, tau)
    z = s0 / (s_max / (S - 1))
    rev = 0.0
    acts = []
    T = len(lam_real)
    for t in range(1, T + 1):
        v = V_all[t]
        lam = float(lam_real[t - 1])
        best, arg = -math.inf, -1
        for a in range(len(p)):
            zn = z + f[a]
            if not (-1e-9 <= zn <= S - 1 + 1e-9):
                continue
            val = lam * (p[a] * tau) + _v_at(v, zn)
            if val > best:
                best, arg = val, a
        rev = rev + lam * (p[arg] * tau)
        z = z + f[arg]
        zr = float(np.rint(z))
        if abs(z - zr) < 1e-9:
            z = zr
        acts.append(arg)
    return rev, z, np.array(acts, np.int32)


# --------------------------------------------------------------------------
# Monte Carlo forward simulation of a policy
# --------------------------------------------------------------------------

def mc_simulate(inst, policy: np.ndarray, n_paths: int, seed: int = 0):
    """Simulate the storage under `policy` [T,M,N,K] along sampled price
    paths; returns (mean, standard error) of the realised total value
    (stage payoffs plus the terminal value)."""
    rng = np.random.default_rng(seed)
    K, T = inst.K, inst.T
    delta = inst.delta
    mu0 = inst.mu0.astype(np.float64)
    k = rng.choice(K, size=n_paths, p=mu0 / mu0.sum())
    s = np.full(n_paths, inst.s0, np.int64)
    m = np.zeros(n_paths, np.int64)
    total = np.zeros(n_paths)
    price = inst.price.astype(np.float64)
    cost = inst.cost.astype(np.float64)
    for t in range(T):
        a = policy[t, m, s, k].astype(np.int64)
        d = a - inst.D_dis
        # grid energy: storage energy times eta_d when discharging, divided
        # by eta_c when charging
        grid = np.where(d < 0, -d * delta * inst.eta_d, np.where(d > 0, -d * delta / inst.eta_c, 0.0))
        r = price[t, k] * grid - cost[a]
        if inst.n_modes == 2:
            r = r - inst.switch_cost * ((m == 1) & (d < 0))
            m = np.where(d < 0, 0, np.where(d > 0, 1, m))
        total += r
        s = s + d
        assert s.min() >= 0 and s.max() < inst.N
        cum = np.cumsum(inst.trans[t].astype(np.float64), axis=1)
        cum[:, -1] = np.inf
        u = rng.random(n_paths)
        k = (u[:, None] > cum[k]).sum(axis=1)
    total += inst.terminal.astype(np.float64)[m, s, k]
    return float(total.mean()), float(total.std(ddof=1) / math.sqrt(n_paths))
