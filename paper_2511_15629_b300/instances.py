"""Seeded synthetic storage-arbitrage instances.

This module only *describes problems*: storage sizes, grids, price processes,
transition matrices, per-action costs and terminal values.  It holds none of
the dynamic-programming arithmetic (no Bellman step, no expectation, no hull);
both the FP64 oracle and the CUDA library consume the arrays it returns.

Every array is rounded to float32 so that the oracle (which promotes them to
float64) and the GPU solve exactly the same instance.

Conventions (shared by the oracle and the library):

* stages ``t = 1..T`` are stored at index ``t-1``;
* SoC grid ``s = 0..N-1`` with step ``delta = s_max / (N-1)`` (Sec. III-A,
  eq. 12);
* actions ``a = 0..A-1`` shift the SoC by ``a - D_dis`` grid steps, so
  ``a < D_dis`` discharges and ``a > D_dis`` charges (the integer
  "recombining" interior of the action grid of eq. 13);
* ``price[t, k]`` is the price of Markov price state ``k`` at stage ``t``;
  ``trans[t, k, k2]`` is the probability of moving from state ``k`` at stage
  ``t`` to ``k2`` at stage ``t+1`` (a Markov generalisation of the
  stagewise-independent price samples of eq. 14);
* ``cost[a]`` is a per-action cost in $ per stage (degradation), given as data;
* ``terminal[m, s, k]`` is the value of ending in SoC ``s``, mode ``m``,
  price state ``k`` (eq. 6 uses zero);
* ``n_modes == 2`` adds a charge->discharge switch flag to the state and a
  fixed ``switch_cost`` paid when discharging right after charging.

The price processes follow Tauchen (1986): an AR(1) log-price deviation
``x_{t+1} = phi x_t + eps``, ``eps ~ N(0, sigma^2)``, discretised on ``K``
equally spaced nodes spanning +-3 unconditional standard deviations.  They
stand in for the ISO-NE real-time price forecasts of Sec. IV, which are not
available.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np
from scipy.special import ndtr

F32 = np.float32


@dataclasses.dataclass
class Instance:
    """One storage asset with its price process (all arrays float32)."""

    name: str
    T: int
    N: int
    K: int
    A: int
    D_dis: int
    D_chg: int
    n_modes: int
    s_max: float       # MWh
    tau: float         # stage length in hours
    eta_c: float       # charge efficiency
    eta_d: float       # discharge efficiency
    switch_cost: float # $ per charge->discharge switch (n_modes == 2)
    price: np.ndarray     # [T, K]
    trans: np.ndarray     # [T, K, K]
    cost: np.ndarray      # [A]
    terminal: np.ndarray  # [n_modes, N, K]
    s0: int = 0
    mu0: Optional[np.ndarray] = None  # [K], initial price-state distribution
    policy_bytes: int = 4
    ckpt_every: int = 0
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def delta(self) -> float:
        return self.s_max / (self.N - 1)

    @property
    def p_max(self) -> float:
        """Storage-side power limit implied by the action band (MW)."""
        return max(self.D_dis, self.D_chg) * self.delta / self.tau

    @property
    def evals(self) -> int:
        """Bellman action evaluations of one sweep: T * n_modes*N * K * A."""
        return self.T * self.n_modes * self.N * self.K * self.A

    def __post_init__(self):
        if self.mu0 is None:
            self.mu0 = np.full(self.K, 1.0 / self.K, dtype=F32)
        assert self.A == self.D_dis + self.D_chg + 1
        for name in ("price", "trans", "cost", "terminal", "mu0"):
            arr = getattr(self, name)
            assert arr.dtype == F32, name
            setattr(self, name, np.ascontiguousarray(arr))
        assert self.price.shape == (self.T, self.K)
        assert self.trans.shape == (self.T, self.K, self.K)
        assert self.cost.shape == (self.A,)
        assert self.terminal.shape == (self.n_modes, self.N, self.K)
        assert self.mu0.shape == (self.K,)


# --------------------------------------------------------------------------
# price processes
# --------------------------------------------------------------------------

def tauchen(K: int, phi: float, sigma: float, m: float = 3.0):
    """Tauchen (1986) discretisation of x' = phi x + N(0, sigma^2).

    Returns (nodes[K], transition[K, K]) in float64; rows sum to 1.
    """
    if K == 1:
        return np.zeros(1), np.ones((1, 1))
    sx = sigma / math.sqrt(1.0 - phi * phi)
    x = np.linspace(-m * sx, m * sx, K)
    w = x[1] - x[0]
    mean = phi * x[:, None]
    upper = ndtr((x[None, :] + w / 2 - mean) / sigma)
    lower = ndtr((x[None, :] - w / 2 - mean) / sigma)
    P = upper - lower
    P[:, 0] = upper[:, 0]
    P[:, -1] = 1.0 - lower[:, -1]
    P = np.maximum(P, 0.0)
    P /= P.sum(axis=1, keepdims=True)
    return x, P


def daily_profile(T: int, tau: float, base: float = 40.0, amp: float = 12.0,
                  evening: float = 10.0) -> np.ndarray:
    """Mean price by stage: a daily sinusoid plus an evening peak ($/MWh)."""
    h = (np.arange(T) * tau) % 24.0
    return (base + amp * np.sin(2 * np.pi * (h - 7.0) / 24.0)
            + evening * np.exp(-((h - 18.5) / 1.5) ** 2))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(F32))


def _renorm_rows_f32(P: np.ndarray) -> np.ndarray:
    """Round a row-stochastic float64 array to float32 (rows stay ~1)."""
    P = np.maximum(P, 0.0)
    P = P / P.sum(axis=-1, keepdims=True)
    return _f32(P)


def _shifts(A: int, D_dis: int) -> np.ndarray:
    return np.arange(A) - D_dis


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def config1(seed: int = 1001) -> Instance:
    """Plain single asset: T=24 hourly, N=101 (1 MWh, step 0.01), A=51, K=5.

    Tauchen phi=0.8, sigma=0.3 around 40 +- 15 sinusoid; -$20 on the lowest
    node in 3 seed-chosen hours; eta 0.95/0.95; $5/MWh on discharged
    (grid-side) energy; zero terminal value; s0 = 50, uniform initial state.
    """
    rng = np.random.default_rng(seed)
    T, N, K, A = 24, 101, 5, 51
    D = 25
    s_max, tau, eta_c, eta_d = 1.0, 1.0, 0.95, 0.95
    x, Pm = tauchen(K, 0.8, 0.3)
    mu = 40.0 + 15.0 * np.sin(2 * np.pi * np.arange(T) / 24.0)
    price = mu[:, None] * np.exp(x)[None, :]
    neg_hours = rng.choice(T, size=3, replace=False)
    price[neg_hours, 0] -= 20.0
    trans = np.broadcast_to(Pm, (T, K, K))
    delta = s_max / (N - 1)
    sh = _shifts(A, D)
    # degradation: $5 per MWh of grid-side discharged energy
    cost = np.where(sh < 0, 5.0 * (-sh) * delta * eta_d, 0.0)
    return Instance("config1", T, N, K, A, D, D, 1, s_max, tau, eta_c, eta_d,
                    0.0, _f32(price), _renorm_rows_f32(trans), _f32(cost),
                    np.zeros((1, N, K), F32), s0=50,
                    meta={"seed": seed, "neg_hours": sorted(int(h) for h in neg_hours)})


def config2(seed: int = 1002) -> Instance:
    """5-minute real-time-shaped asset with a charge->discharge switch cost.

    T=288, 4 MWh on N=1001 (step 0.004), A=201 (+-100 steps), eta 0.92/0.95,
    K=20 = 19 Tauchen nodes (phi=0.95, sigma=0.25) + 1 spike node at 5x the
    median price entered with probability 0.02 from every row; a 6-hour
    (72-stage) stretch whose lowest 4 nodes are below -$30; $50 per
    charge->discharge switch via a 2-valued mode flag.
    """
    rng = np.random.default_rng(seed)
    T, N, K, A, D = 288, 1001, 20, 201, 100
    s_max, tau, eta_c, eta_d = 4.0, 1.0 / 12.0, 0.92, 0.95
    Kt = K - 1
    x, Pm = tauchen(Kt, 0.95, 0.25)
    mu = daily_profile(T, tau)
    price = np.empty((T, K))
    price[:, :Kt] = mu[:, None] * np.exp(x)[None, :]
    med = Kt // 2
    price[:, Kt] = 5.0 * price[:, med]
    start = int(rng.integers(0, T - 72))
    for j in range(4):
        price[start:start + 72, j] = -31.0 - 2.0 * (3 - j) - rng.uniform(0, 1, 72)
    P = np.zeros((K, K))
    P[:Kt, :Kt] = 0.98 * Pm
    P[:Kt, Kt] = 0.02
    P[Kt, :Kt] = 0.98 * Pm[med]
    P[Kt, Kt] = 0.02
    trans = np.broadcast_to(P, (T, K, K))
    return Instance("config2", T, N, K, A, D, D, 2, s_max, tau, eta_c, eta_d,
                    50.0, _f32(price), _renorm_rows_f32(trans),
                    np.zeros(A, F32), np.zeros((2, N, K), F32), s0=N // 2,
                    meta={"seed": seed, "negative_stretch": [start, start + 72]})


def config3(seed: int = 1003) -> Instance:
    """Large asset: T=2016 5-minute stages, N=5001, A=201, K=64.

    Dense transition matrices drawn fresh per stage: rows are
    0.5 * Dirichlet(alpha=0.5) + 0.5 * Tauchen (phi=0.9, sigma=0.3) row.
    Piecewise-quadratic degradation cost on the storage-side energy moved in
    a stage, x = |shift| * delta:  c = 3 x + 200 max(x - 0.1, 0)^2.
    Terminal value V_{T+1}(s) = 30 $/MWh * s.
    """
    rng = np.random.default_rng(seed)
    T, N, K, A, D = 2016, 5001, 64, 201, 100
    s_max, tau, eta_c, eta_d = 10.0, 1.0 / 12.0, 0.93, 0.96
    x, Pm = tauchen(K, 0.9, 0.3)
    mu = daily_profile(T, tau)
    price = mu[:, None] * np.exp(x)[None, :]
    dirich = rng.gamma(0.5, size=(T, K, K))
    dirich /= dirich.sum(axis=2, keepdims=True)
    trans = 0.5 * dirich + 0.5 * Pm[None]
    delta = s_max / (N - 1)
    xs = np.abs(_shifts(A, D)) * delta
    cost = 3.0 * xs + 200.0 * np.maximum(xs - 0.1, 0.0) ** 2
    soc = np.arange(N) * delta
    terminal = np.broadcast_to((30.0 * soc)[None, :, None], (1, N, K))
    return Instance("config3", T, N, K, A, D, D, 1, s_max, tau, eta_c, eta_d,
                    0.0, _f32(price), _renorm_rows_f32(trans), _f32(cost),
                    _f32(terminal), s0=N // 2, meta={"seed": seed})


def config4_asset(j: int) -> Instance:
    """Asset j of the 256-asset heterogeneous portfolio (seed 4000 + j).

    N ~ U{201..4001}; duration 1-8 h at 1 MW nominal, so s_max = duration;
    5-minute stages (T=288); A odd in [41, 401]; K ~ U{8..40}; efficiencies
    in [0.85, 0.97]; per-asset Tauchen AR(1) with phi in [0.7, 0.97],
    sigma in [0.1, 0.4]; 0-5% of price nodes shifted negative.
    """
    rng = np.random.default_rng(4000 + j)
    T = 288
    N = int(rng.integers(201, 4002))
    dur = float(rng.uniform(1.0, 8.0))
    A = 2 * int(rng.integers(20, 201)) + 1
    K = int(rng.integers(8, 41))
    eta_c = float(rng.uniform(0.85, 0.97))
    eta_d = float(rng.uniform(0.85, 0.97))
    phi = float(rng.uniform(0.7, 0.97))
    sigma = float(rng.uniform(0.1, 0.4))
    neg_frac = float(rng.uniform(0.0, 0.05))
    tau = 1.0 / 12.0
    D = (A - 1) // 2
    x, Pm = tauchen(K, phi, sigma)
    mu = daily_profile(T, tau, base=float(rng.uniform(30, 50)))
    price = mu[:, None] * np.exp(x)[None, :]
    n_neg = int(rng.binomial(K, neg_frac))
    if n_neg:
        price[:, :n_neg] = -rng.uniform(5.0, 40.0, size=(T, n_neg))
    trans = np.broadcast_to(Pm, (T, K, K))
    delta = dur / (N - 1)
    sh = _shifts(A, D)
    cost = np.where(sh < 0, 5.0 * (-sh) * delta * eta_d, 0.0)
    return Instance(f"config4_asset{j}", T, N, K, A, D, D, 1, dur, tau,
                    eta_c, eta_d, 0.0, _f32(price), _renorm_rows_f32(trans),
                    _f32(cost), np.zeros((1, N, K), F32), s0=N // 2,
                    meta={"seed": 4000 + j, "phi": phi, "sigma": sigma,
                          "n_neg": n_neg})


def config4(n_assets: int = 256) -> List[Instance]:
    """The heterogeneous portfolio (first ``n_assets`` of the 256)."""
    return [config4_asset(j) for j in range(n_assets)]


def config5(seed: int = 1005) -> Instance:
    """Adjoint workload: T=288, N=2001, A=201, K=32, int16 policy,
    checkpoints every 32 stages, s0 = 1000 (50%), uniform initial state."""
    rng = np.random.default_rng(seed)
    T, N, K, A, D = 288, 2001, 32, 201, 100
    s_max, tau, eta_c, eta_d = 4.0, 1.0 / 12.0, 0.95, 0.95
    x, Pm = tauchen(K, 0.9, 0.3)
    mu = daily_profile(T, tau) * rng.uniform(0.97, 1.03, size=T)
    price = mu[:, None] * np.exp(x)[None, :]
    trans = np.broadcast_to(Pm, (T, K, K))
    delta = s_max / (N - 1)
    sh = _shifts(A, D)
    cost = np.where(sh < 0, 5.0 * (-sh) * delta * eta_d, 0.0)
    return Instance("config5", T, N, K, A, D, D, 1, s_max, tau, eta_c, eta_d,
                    0.0, _f32(price), _renorm_rows_f32(trans), _f32(cost),
                    np.zeros((1, N, K), F32), s0=1000, policy_bytes=2,
                    ckpt_every=32, meta={"seed": seed})


CONFIGS = {1: config1, 2: config2, 3: config3, 5: config5}


# --------------------------------------------------------------------------
# generic random instances for tests (ragged shapes, ties, negative prices)
# --------------------------------------------------------------------------

def random_instance(seed: int, T: int, N: int, K: int, D_dis: int, D_chg: int,
                    n_modes: int = 1, *, neg_prob: float = 0.1,
                    switch_cost: float = 7.0, terminal: str = "random",
                    dirichlet: bool = True, eta=(0.9, 0.93), s_max: float = None,
                    tau: float = 1.0, cost: str = "linear",
                    integer_prices: bool = False) -> Instance:
    """A small random instance for parity and property tests."""
    rng = np.random.default_rng(seed)
    A = D_dis + D_chg + 1
    if s_max is None:
        s_max = 0.05 * (N - 1)
    if integer_prices:
        price = rng.integers(-10, 60, size=(T, K)).astype(np.float64)
    else:
        price = rng.uniform(5.0, 80.0, size=(T, K))
        neg = rng.random((T, K)) < neg_prob
        price[neg] = -rng.uniform(0.0, 30.0, size=int(neg.sum()))
    if dirichlet and K > 1:
        trans = rng.dirichlet(np.full(K, 0.7), size=(T, K))
    else:
        _, Pm = tauchen(K, 0.8, 0.3)
        trans = np.broadcast_to(Pm, (T, K, K))
    delta = s_max / (N - 1)
    sh = _shifts(A, D_dis)
    if cost == "linear":
        c = np.where(sh < 0, 2.0 * (-sh) * delta, 0.0)
    elif cost == "zero":
        c = np.zeros(A)
    elif cost == "nonconvex":
        c = rng.uniform(0.0, 3.0, size=A)
        c[D_dis] = 0.0
    else:
        raise ValueError(cost)
    if terminal == "random":
        term = rng.uniform(0.0, 20.0, size=(n_modes, N, K))
    elif terminal == "zero":
        term = np.zeros((n_modes, N, K))
    elif terminal == "linear":
        soc = np.arange(N) * delta
        term = np.broadcast_to((25.0 * soc)[None, :, None], (n_modes, N, K))
    else:
        raise ValueError(terminal)
    return Instance(f"random{seed}", T, N, K, A, D_dis, D_chg, n_modes, s_max,
                    tau, float(eta[0]), float(eta[1]),
                    switch_cost if n_modes == 2 else 0.0, _f32(price),
                    _renorm_rows_f32(trans), _f32(c), _f32(term),
                    s0=int(rng.integers(0, N)), meta={"seed": seed})


def iid_instance(seed: int, T: int, N: int, R: int, D_dis: int, D_chg: int,
                 **kw) -> Instance:
    """Stagewise-independent prices (the paper's setting, eq. 14): every row
    of trans[t] is the probability vector of the stage-(t+1) price samples."""
    inst = random_instance(seed, T, N, R, D_dis, D_chg, **kw)
    rng = np.random.default_rng(seed + 7)
    pis = _renorm_rows_f32(rng.dirichlet(np.full(R, 1.0), size=T + 1))
    # stage-t price samples have probabilities pis[t-1]; from any state at
    # stage t the chain moves to stage-(t+1) sample k2 with pis[t][k2]
    inst.trans = np.ascontiguousarray(np.broadcast_to(pis[1:, None, :], (T, R, R)).copy())
    inst.mu0 = np.ascontiguousarray(pis[0].copy())
    inst.meta["pi_hat"] = pis
    return inst


# --------------------------------------------------------------------------
# The paper's own setting: stagewise-independent price samples, eq. 13 grid
# --------------------------------------------------------------------------

@dataclasses.dataclass
class IidProblem:
    """Algorithm 1 input: R price samples (lam_hat, pi_hat) per stage for a
    storage of s_max MWh on an S-point SoC grid with power limit p_max and the
    single efficiency eta of eq. 2; hourly stages by default."""
    name: str
    T: int
    S: int
    R: int
    s_max: float
    p_max: float
    eta: float
    lam_hat: np.ndarray      # [T, R] float32, $/MWh
    pi_hat: np.ndarray       # [T, R] float32, rows sum to 1 (rounded)
    tau: float = 1.0
    terminal: Optional[np.ndarray] = None   # [S] float32 or None (zero, as in the paper)
    policy_bytes: int = 0

    @property
    def delta(self) -> float:
        return self.s_max / (self.S - 1)


def iid_problem(seed: int, T: int, S: int, R: int, hours: float, *, p_max: float = 1.0,
                eta: float = math.sqrt(0.85), neg_prob: float = 0.03,
                weights: str = "uniform", terminal: bool = False,
                name: str = "iid") -> IidProblem:
    """Synthetic stand-in for the paper's real-time price samples (Sec. IV):
    per stage R samples around a daily mean profile (40 +- 15 $/MWh with an
    evening peak), lognormal spread sigma 0.35, a few negative prices
    (probability neg_prob, down to -$30), uniform sample weights (as the
    paper's empirical samples) or Dirichlet ones.  s_max = hours * p_max."""
    rng = np.random.default_rng(seed)
    h = np.arange(T) % 24
    mean = 40.0 + 15.0 * np.sin(2 * np.pi * (h - 9) / 24.0) + 10.0 * np.exp(-0.5 * ((h - 18) / 2.0) ** 2)
    lam = mean[:, None] * np.exp(rng.normal(0.0, 0.35, size=(T, R)) - 0.5 * 0.35 ** 2)
    neg = rng.random((T, R)) < neg_prob
    lam = np.where(neg, -rng.uniform(0.0, 30.0, size=(T, R)), lam)
    if weights == "uniform":
        pi = np.full((T, R), 1.0 / R)
    else:
        pi = rng.dirichlet(np.full(R, 1.0), size=T)
    term = None
    if terminal:
        term = (25.0 * np.linspace(0.0, hours * p_max, S)).astype(np.float32)
    return IidProblem(name, T, S, R, float(hours * p_max), float(p_max), float(eta),
                      np.ascontiguousarray(lam.astype(np.float32)),
                      _renorm_rows_f32(pi), terminal=term)


# The six storage/grid combinations of the paper's runtime study (Table III):
# (duration hours, S, P) with p_max = 1 MW, eta = sqrt(0.85), R = 200 samples,
# T = 8784 hourly stages.
TABLE3_CASES = [(4, 41, 22), (20, 201, 22), (100, 1001, 22), (4, 401, 203), (20, 2001, 203),
                (100, 10001, 203)]


def table3_problem(case: int, seed: int = 3000, T: int = 8784, R: int = 200) -> IidProblem:
    hours, S, _ = TABLE3_CASES[case]
    return iid_problem(seed + case, T, S, R, hours, name=f"table3-{hours}h-S{S}")
