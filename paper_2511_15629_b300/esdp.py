"""Thin ctypes binding of the C ABI in include/esdp.h (libesdp.so).

Argument marshalling only: every step of the solve, the bid curves and the
adjoint runs in the CUDA library.  There is no fallback: if the library is
missing or the device is absent the calls raise.

Two calling conventions, chosen per context:
  * host mode (default): numpy float32 arrays in and out, calls block;
  * device mode (``device_ptrs=True``): torch CUDA tensors (or raw device
    addresses), work queued on the given stream (default: torch's current
    stream).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libesdp.so")
# measurement build of the same sources (per-phase sweep clock counters)
LIB_PHASE_PATH = os.path.join(_HERE, "libesdp_phase.so")

ESDP_OK = 0
ESDP_EINVAL = -1
ESDP_ENOMEM = -2
ESDP_ECUDA = -3
ESDP_ETIMEOUT = -4
ESDP_ESTATE = -5
ESDP_ENUMERIC = -6

ESDP_DEVICE_PTRS = 1
ESDP_KEEP_EV = 2
ESDP_CHECK_ROWS = 4
ESDP_NO_VALIDATE = 8
ESDP_TIME_SWEEP = 16

EXPORTS = ["esdp_create", "esdp_solve", "esdp_policy", "esdp_expected_value", "esdp_bid_curves",
           "esdp_bids_at", "esdp_bid_curves_packed",
           "esdp_objective", "esdp_grad", "esdp_iid_actions", "esdp_solve_iid", "esdp_iid_bids",
           "esdp_iid_clear", "esdp_iid_last_sweep_ms", "esdp_autotune", "esdp_alu_probe",
           "esdp_status", "esdp_sweep_ms", "esdp_phase_clocks", "esdp_launch_info", "esdp_destroy", "esdp_last_error",
           "esdp_version"]


class EsdpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"esdp error {code}: {msg}")
        self.code = code


class Asset(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("N", ctypes.c_int32), ("K", ctypes.c_int32),
                ("A", ctypes.c_int32), ("D_dis", ctypes.c_int32), ("D_chg", ctypes.c_int32),
                ("n_modes", ctypes.c_int32), ("policy_bytes", ctypes.c_int32),
                ("ckpt_every", ctypes.c_int32), ("s0", ctypes.c_int32),
                ("s_max", ctypes.c_double), ("tau", ctypes.c_double), ("eta_c", ctypes.c_double),
                ("eta_d", ctypes.c_double), ("switch_cost", ctypes.c_double)]


_lib = None


def load_library(path: Optional[str] = None):
    """Load libesdp.so, or the library at `path` (the phase-clock build),
    once per process; raises if it has not been built."""
    global _lib
    if _lib is not None:
        if path is not None and getattr(_lib, "_esdp_path", LIB_PATH) != path:
            raise RuntimeError(f"{_lib._esdp_path} is already loaded")
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_2511_15629_b300.build`")
    lib = ctypes.CDLL(path)
    lib._esdp_path = path
    vp = ctypes.c_void_p
    i32 = ctypes.c_int32
    lib.esdp_create.argtypes = [ctypes.POINTER(Asset), i32, ctypes.c_uint32, ctypes.POINTER(vp)]
    lib.esdp_solve.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.esdp_policy.argtypes = [vp, i32, i32, vp, vp]
    lib.esdp_expected_value.argtypes = [vp, i32, i32, vp, vp]
    lib.esdp_bid_curves.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp]
    lib.esdp_bids_at.argtypes = [vp, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.esdp_bid_curves_packed.argtypes = [vp, i32, i32, i32, vp, vp, vp, ctypes.c_int64, vp]
    lib.esdp_objective.argtypes = [vp, i32, vp, vp, vp]
    lib.esdp_grad.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.esdp_autotune.argtypes = [vp, vp]
    lib.esdp_status.argtypes = [vp, vp]
    lib.esdp_sweep_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    lib.esdp_phase_clocks.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i32]
    lib.esdp_launch_info.argtypes = [vp] + [ctypes.POINTER(i32)] * 7
    lib.esdp_destroy.argtypes = [vp]
    lib.esdp_destroy.restype = None
    lib.esdp_last_error.argtypes = [vp]
    lib.esdp_last_error.restype = ctypes.c_char_p
    lib.esdp_version.argtypes = []
    lib.esdp_alu_probe.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), vp]
    lib.esdp_iid_last_sweep_ms.argtypes = []
    for name in EXPORTS:
        if name not in ("esdp_destroy", "esdp_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    lib.esdp_iid_last_sweep_ms.restype = ctypes.c_double
    _lib = lib
    return lib


def asset_from_instance(inst) -> Asset:
    return Asset(T=inst.T, N=inst.N, K=inst.K, A=inst.A, D_dis=inst.D_dis, D_chg=inst.D_chg,
                 n_modes=inst.n_modes, policy_bytes=inst.policy_bytes,
                 ckpt_every=inst.ckpt_every, s0=inst.s0, s_max=inst.s_max, tau=inst.tau,
                 eta_c=inst.eta_c, eta_d=inst.eta_d, switch_cost=inst.switch_cost)


def concat_inputs(instances: Sequence) -> dict:
    """Concatenate the per-asset float32 inputs in asset order."""
    cat = lambda name: np.ascontiguousarray(
        np.concatenate([getattr(i, name).ravel() for i in instances]).astype(np.float32))
    return {"price": cat("price"), "trans": cat("trans"), "cost": cat("cost"),
            "terminal": cat("terminal")}


def _host_ptr(a: Optional[np.ndarray], dtype) -> Optional[int]:
    if a is None:
        return None
    assert isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous, \
        "expected a C-contiguous numpy array of " + str(dtype)
    return a.ctypes.data


def _dev_ptr(a) -> Optional[int]:
    if a is None:
        return None
    if isinstance(a, int):
        return a
    assert a.is_cuda and a.is_contiguous(), "expected a contiguous CUDA tensor"
    return a.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Solver:
    """One esdp context over a list of assets (instances)."""

    def __init__(self, instances: Sequence, *, device_ptrs: bool = False, keep_ev: bool = False,
                 check_rows: bool = False, no_validate: bool = False, time_sweep: bool = False):
        self._lib = load_library()
        self.instances = list(instances)
        self.device = device_ptrs
        flags = ((ESDP_DEVICE_PTRS if device_ptrs else 0) | (ESDP_KEEP_EV if keep_ev else 0)
                 | (ESDP_CHECK_ROWS if check_rows else 0) | (ESDP_NO_VALIDATE if no_validate else 0)
                 | (ESDP_TIME_SWEEP if time_sweep else 0))
        arr = (Asset * len(self.instances))(*[asset_from_instance(i) for i in self.instances])
        self._ctx = ctypes.c_void_p()
        rc = self._lib.esdp_create(arr, len(self.instances), flags, ctypes.byref(self._ctx))
        if rc != ESDP_OK:
            msg = self.last_error()
            self.close()
            raise EsdpError(rc, msg)

    # -- helpers ---------------------------------------------------------
    def last_error(self) -> str:
        if not self._ctx:
            return "no context"
        return self._lib.esdp_last_error(self._ctx).decode()

    def _check(self, rc: int):
        if rc != ESDP_OK:
            raise EsdpError(rc, self.last_error())

    def _ptr(self, a, dtype=np.float32):
        return _dev_ptr(a) if self.device else _host_ptr(a, dtype)

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.esdp_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API -------------------------------------------------------------
    def solve(self, price, trans, cost, terminal, V1=None, stream=None):
        self._check(self._lib.esdp_solve(self._ctx, self._ptr(price), self._ptr(trans),
                                         self._ptr(cost), self._ptr(terminal), self._ptr(V1),
                                         _stream(stream)))
        return V1

    def solve_instances(self, V1: Optional[np.ndarray] = None) -> np.ndarray:
        """Host mode: solve the context's own instances, return V1 per asset."""
        assert not self.device
        cat = concat_inputs(self.instances)
        n = sum(i.n_modes * i.N * i.K for i in self.instances)
        V1 = np.empty(n, np.float32) if V1 is None else V1
        self.solve(cat["price"], cat["trans"], cat["cost"], cat["terminal"], V1)
        out, o = [], 0
        for i in self.instances:
            L = i.n_modes * i.N * i.K
            out.append(V1[o:o + L].reshape(i.n_modes, i.N, i.K))
            o += L
        return out

    def policy(self, asset: int, t: int, out=None, stream=None):
        inst = self.instances[asset]
        if out is None:
            assert not self.device
            dt = np.int16 if inst.policy_bytes == 2 else np.int32
            out = np.empty((inst.n_modes, inst.N, inst.K), dt)
        dtype = out.dtype if isinstance(out, np.ndarray) else None
        p = _dev_ptr(out) if self.device else _host_ptr(out, dtype)
        self._check(self._lib.esdp_policy(self._ctx, asset, t, p, _stream(stream)))
        return out

    def expected_value(self, asset: int, t: int, out=None, stream=None):
        inst = self.instances[asset]
        if out is None:
            assert not self.device
            out = np.empty((inst.n_modes, inst.N, inst.K), np.float32)
        self._check(self._lib.esdp_expected_value(self._ctx, asset, t, self._ptr(out),
                                                  _stream(stream)))
        return out

    def bid_curves(self, asset: int, t0: int, t1: int, n_bp=None, idx=None, slope=None,
                   stream=None):
        inst = self.instances[asset]
        n = t1 - t0
        if n_bp is None:
            assert not self.device
            n_bp = np.empty((n, inst.n_modes, inst.K), np.int32)
            idx = np.empty((n, inst.n_modes, inst.K, inst.N), np.int32)
            slope = np.empty((n, inst.n_modes, inst.K, inst.N), np.float32)
        p = (lambda a, d: _dev_ptr(a)) if self.device else _host_ptr
        self._check(self._lib.esdp_bid_curves(self._ctx, asset, t0, t1, p(n_bp, np.int32),
                                              p(idx, np.int32), p(slope, np.float32),
                                              _stream(stream)))
        return n_bp, idx, slope

    def bid_curves_packed(self, asset: int, t0: int, t1: int, offsets=None, idx=None, slope=None,
                          stream=None):
        """Bid curves without row padding (esdp_bid_curves_packed): envelope h
        owns [offsets[h], offsets[h+1]) of idx and slope.  Host mode allocates
        worst-case arrays when not given and returns views of `total`
        entries; device mode writes the given tensors (cap = their length)."""
        inst = self.instances[asset]
        nh = (t1 - t0) * inst.n_modes * inst.K
        if offsets is None:
            assert not self.device
            offsets = np.empty(nh + 1, np.int64)
            idx = np.empty(nh * inst.N, np.int32)
            slope = np.empty(nh * inst.N, np.float32)
        if self.device:
            cap = min(idx.numel(), slope.numel())
            p = lambda a, d: _dev_ptr(a)
        else:
            cap = min(idx.size, slope.size)
            p = _host_ptr
        self._check(self._lib.esdp_bid_curves_packed(self._ctx, asset, t0, t1,
                                                     p(offsets, np.int64), p(idx, np.int32),
                                                     p(slope, np.float32), cap, _stream(stream)))
        if not self.device:
            total = int(offsets[-1])
            return offsets, idx[:total], slope[:total]
        return offsets, idx, slope

    def bids_at(self, asset: int, t0: int, t1: int, s: int, n_bp, idx, n_pts=None, p_mw=None,
                price=None, stream=None):
        """Price-quantity bids at SoC index s (esdp_bids_at) from the envelopes
        `n_bp`, `idx` of bid_curves over the same stages: (n_pts [n,M,K],
        p_mw [n,M,K,A] MW ascending, price [n,M,K,A] $/MWh of each segment)."""
        inst = self.instances[asset]
        n = t1 - t0
        if n_pts is None:
            assert not self.device
            n_pts = np.empty((n, inst.n_modes, inst.K), np.int32)
            p_mw = np.empty((n, inst.n_modes, inst.K, inst.A), np.float64)
            price = np.empty((n, inst.n_modes, inst.K, inst.A), np.float32)
        if self.device:
            p = lambda a, d: _dev_ptr(a)
        else:
            n_bp = np.ascontiguousarray(n_bp, dtype=np.int32)
            idx = np.ascontiguousarray(idx, dtype=np.int32)
            p = _host_ptr
        self._check(self._lib.esdp_bids_at(self._ctx, asset, t0, t1, s, p(n_bp, np.int32),
                                           p(idx, np.int32), p(n_pts, np.int32),
                                           p(p_mw, np.float64), p(price, np.float32),
                                           _stream(stream)))
        return n_pts, p_mw, price

    def objective(self, asset: int, mu0, J=None, stream=None):
        """J = sum_k mu0[k] V_1[0][s0][k] of the last solve (double)."""
        if not self.device:
            mu0 = np.ascontiguousarray(mu0, dtype=np.float32)
            J = np.zeros(1, np.float64) if J is None else J
            ptr = _host_ptr
        else:
            ptr = lambda a, dt: _dev_ptr(a)
        self._check(self._lib.esdp_objective(self._ctx, asset, ptr(mu0, np.float32),
                                             ptr(J, np.float64), _stream(stream)))
        return J

    def grad(self, asset: int, mu0, J=None, d_price=None, d_trans=None, d_eta=None,
             d_cost=None, d_switch=None, d_terminal=None, d_mu0=None, stream=None, extra=False):
        """Sensitivities of J (esdp_grad).  Host mode allocates the outputs it
        is not given: (J, d_price, d_trans, d_eta), plus (d_cost, d_switch,
        d_terminal, d_mu0) with extra=True.  Device mode writes the tensors it
        is given (None: not computed)."""
        inst = self.instances[asset]
        if not self.device:
            mu0 = np.ascontiguousarray(mu0, dtype=np.float32)
            J = np.zeros(1, np.float64) if J is None else J
            d_price = np.zeros((inst.T, inst.K), np.float32) if d_price is None else d_price
            d_trans = (np.zeros((inst.T, inst.K, inst.K), np.float32) if d_trans is None
                       else d_trans)
            d_eta = np.zeros(2, np.float64) if d_eta is None else d_eta
            if extra:
                d_cost = np.zeros(inst.A, np.float32) if d_cost is None else d_cost
                d_switch = np.zeros(1, np.float64) if d_switch is None else d_switch
                d_terminal = (np.zeros((inst.n_modes, inst.N, inst.K), np.float32)
                              if d_terminal is None else d_terminal)
                d_mu0 = np.zeros(inst.K, np.float32) if d_mu0 is None else d_mu0
            ptr = lambda a, dt: _host_ptr(a, dt)
        else:
            ptr = lambda a, dt: _dev_ptr(a)
        self._check(self._lib.esdp_grad(self._ctx, asset, ptr(mu0, np.float32),
                                        ptr(J, np.float64), ptr(d_price, np.float32),
                                        ptr(d_trans, np.float32), ptr(d_eta, np.float64),
                                        ptr(d_cost, np.float32), ptr(d_switch, np.float64),
                                        ptr(d_terminal, np.float32), ptr(d_mu0, np.float32),
                                        _stream(stream)))
        if extra:
            return J, d_price, d_trans, d_eta, d_cost, d_switch, d_terminal, d_mu0
        return J, d_price, d_trans, d_eta

    def autotune(self, stream=None):
        self._check(self._lib.esdp_autotune(self._ctx, _stream(stream)))

    def status(self, stream=None) -> int:
        return int(self._lib.esdp_status(self._ctx, _stream(stream)))

    PHASES = ("inputs", "neighbour wait", "EV halo copy + level", "max-plus loop",
              "merge + argmax recovery", "EV contraction", "release", "next-stage issue")

    def phase_clocks(self) -> dict:
        """Per-stage cycles of each sweep phase of the last solve (needs the
        library built with phase clocks: load_library(LIB_PHASE_PATH))."""
        out = (ctypes.c_double * 8)()
        self._check(self._lib.esdp_phase_clocks(self._ctx, out, 8))
        return {name: float(v) for name, v in zip(self.PHASES, out)}

    def sweep_ms(self) -> float:
        """Device time (ms) of the last solve's sweep kernel (needs
        time_sweep=True); waits for that launch."""
        ms = ctypes.c_float()
        self._check(self._lib.esdp_sweep_ms(self._ctx, ctypes.byref(ms)))
        return float(ms.value)

    EV_PATHS = {0: "simt", 1: "tcgen05", 2: "mma.sync"}

    def launch_info(self) -> dict:
        vals = [ctypes.c_int32() for _ in range(7)]
        self._check(self._lib.esdp_launch_info(self._ctx, *[ctypes.byref(v) for v in vals]))
        keys = ["grid", "block", "items", "rows_per_tile", "parts", "rows_per_thread"]
        info = {k: v.value for k, v in zip(keys, vals)}
        info["ev"] = self.EV_PATHS.get(vals[6].value, "none")
        return info


class IidProblemC(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("S", ctypes.c_int32), ("R", ctypes.c_int32),
                ("policy_bytes", ctypes.c_int32), ("s_max", ctypes.c_double),
                ("p_max", ctypes.c_double), ("eta", ctypes.c_double), ("tau", ctypes.c_double)]


def _iid_struct(prob, policy_bytes=None) -> IidProblemC:
    pb = prob.policy_bytes if policy_bytes is None else policy_bytes
    return IidProblemC(prob.T, prob.S, prob.R, pb, prob.s_max, prob.p_max, prob.eta, prob.tau)


def iid_actions(prob) -> np.ndarray:
    """The power levels of eq. 13 (esdp_iid_actions), MW ascending."""
    lib = load_library()
    fn = lib.esdp_iid_actions
    fn.argtypes = [ctypes.POINTER(IidProblemC), ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
    fn.restype = ctypes.c_int
    q = _iid_struct(prob, 0)
    n = ctypes.c_int32()
    rc = fn(ctypes.byref(q), None, ctypes.byref(n))
    if rc != ESDP_OK:
        raise EsdpError(rc, "invalid problem")
    out = np.empty(n.value, np.float64)
    fn(ctypes.byref(q), out.ctypes.data, ctypes.byref(n))
    return out


def solve_iid(prob, V0=None, policy=None, *, device=False, lam_hat=None, pi_hat=None,
              terminal=None, policy_bytes=None, V_all=None, keep_values=False, stream=None):
    """Algorithm 1 on the GPU (esdp_solve_iid).  Host mode (default): numpy
    in and out, returns V0 [S], then the policy [T,S,R] when policy_bytes > 0
    and V_all [T+1,S] (V_t of every stage) with keep_values.  Device mode:
    torch CUDA tensors (or raw device addresses) for lam_hat, pi_hat,
    terminal, V0, V_all and policy."""
    lib = load_library()
    fn = lib.esdp_solve_iid
    fn.argtypes = [ctypes.POINTER(IidProblemC)] + [ctypes.c_void_p] * 6 + \
        [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int32]
    fn.restype = ctypes.c_int
    q = _iid_struct(prob, policy_bytes)
    err = ctypes.create_string_buffer(512)
    if device:
        rc = fn(ctypes.byref(q), _dev_ptr(lam_hat), _dev_ptr(pi_hat), _dev_ptr(terminal),
                _dev_ptr(V0), _dev_ptr(V_all), _dev_ptr(policy), ESDP_DEVICE_PTRS, _stream(stream),
                err, len(err))
    else:
        lam = np.ascontiguousarray(prob.lam_hat if lam_hat is None else lam_hat, np.float32)
        pi = np.ascontiguousarray(prob.pi_hat if pi_hat is None else pi_hat, np.float32)
        term = prob.terminal if terminal is None else terminal
        term = None if term is None else np.ascontiguousarray(term, np.float32)
        V0 = np.empty(prob.S, np.float32) if V0 is None else V0
        if q.policy_bytes and policy is None:
            policy = np.empty((prob.T, prob.S, prob.R), np.int16 if q.policy_bytes == 2 else np.int32)
        if keep_values and V_all is None:
            V_all = np.empty((prob.T + 1, prob.S), np.float32)
        rc = fn(ctypes.byref(q), lam.ctypes.data, pi.ctypes.data,
                None if term is None else term.ctypes.data, V0.ctypes.data,
                None if V_all is None else V_all.ctypes.data,
                None if policy is None else policy.ctypes.data, 0, _stream(stream), err, len(err))
    if rc != ESDP_OK:
        raise EsdpError(rc, err.value.decode())
    out = (V0,)
    if q.policy_bytes:
        out += (policy,)
    if keep_values and not device:
        out += (V_all,)
    return out if len(out) > 1 else V0


def iid_last_sweep_ms() -> float:
    """Device time (ms, CUDA events) of the sweep of this thread's last
    successful solve_iid, without its workspace set-up; negative before any."""
    return float(load_library().esdp_iid_last_sweep_ms())


def iid_bids(prob, V_all, t0: int, t1: int, stream=None):
    """Convexified bid curves (esdp_iid_bids) of delivery intervals t0..t1-1
    for every grid SoC, from V_all [T+1,S] on the device (torch).  Returns
    torch tensors n_bp [n,S], bp_action [n,S,P], bp_price [n,S,P]."""
    import torch
    lib = load_library()
    fn = lib.esdp_iid_bids
    fn.argtypes = [ctypes.POINTER(IidProblemC), ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32] + \
        [ctypes.c_void_p] * 4 + [ctypes.c_char_p, ctypes.c_int32]
    fn.restype = ctypes.c_int
    q = _iid_struct(prob, 0)
    P = len(iid_actions(prob))
    n = t1 - t0
    dev = V_all.device
    n_bp = torch.empty((n, prob.S), dtype=torch.int32, device=dev)
    act = torch.empty((n, prob.S, P), dtype=torch.int32, device=dev)
    price = torch.empty((n, prob.S, P), dtype=torch.float32, device=dev)
    err = ctypes.create_string_buffer(512)
    rc = fn(ctypes.byref(q), _dev_ptr(V_all), t0, t1, _dev_ptr(n_bp), _dev_ptr(act),
            _dev_ptr(price), _stream(stream), err, len(err))
    if rc != ESDP_OK:
        raise EsdpError(rc, err.value.decode())
    return n_bp, act, price


def iid_clear(prob, V_all, lam_real, s0: float, keep_actions: bool = True, stream=None):
    """Merit-order clearing (esdp_iid_clear) of the price paths lam_real
    [n_paths,T] (torch, device) from SoC s0 (MWh).  Returns torch tensors
    revenue [n_paths] (double), s_end [n_paths] (grid steps) and the actions
    [n_paths,T] (or None)."""
    import torch
    lib = load_library()
    fn = lib.esdp_iid_clear
    fn.argtypes = [ctypes.POINTER(IidProblemC), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                   ctypes.c_double] + [ctypes.c_void_p] * 4 + [ctypes.c_char_p, ctypes.c_int32]
    fn.restype = ctypes.c_int
    q = _iid_struct(prob, 0)
    n_paths = lam_real.shape[0]
    dev = lam_real.device
    rev = torch.empty(n_paths, dtype=torch.float64, device=dev)
    s_end = torch.empty(n_paths, dtype=torch.float64, device=dev)
    act = torch.empty((n_paths, prob.T), dtype=torch.int32, device=dev) if keep_actions else None
    err = ctypes.create_string_buffer(512)
    rc = fn(ctypes.byref(q), _dev_ptr(V_all), _dev_ptr(lam_real), n_paths, float(s0),
            _dev_ptr(rev), _dev_ptr(s_end), _dev_ptr(act), _stream(stream), err, len(err))
    if rc != ESDP_OK:
        raise EsdpError(rc, err.value.decode())
    return rev, s_end, act


def solve_noalloc(inst, price, trans, cost, terminal, V1, policy=None, stream=None) -> None:
    """Allocation-free solve of one asset (esdp_solve_noalloc): for callers
    that cannot allocate device memory.  All arrays are device tensors (or
    raw device addresses) that the caller owns; the library's fixed device
    workspace is shared by every call on the device, so overlapping calls
    must be serialised.  Blocks until the solve has finished."""
    lib = load_library()
    fn = lib.esdp_solve_noalloc
    fn.argtypes = [ctypes.POINTER(Asset)] + [ctypes.c_void_p] * 8 + [ctypes.c_int32]
    fn.restype = ctypes.c_int
    a = asset_from_instance(inst)
    err = ctypes.create_string_buffer(512)
    rc = fn(ctypes.byref(a), _dev_ptr(price), _dev_ptr(trans), _dev_ptr(cost), _dev_ptr(terminal),
            _dev_ptr(V1), _dev_ptr(policy), _stream(stream), err, len(err))
    if rc != ESDP_OK:
        raise EsdpError(rc, err.value.decode())


ALU_PROBE_KINDS = ("add.f32", "add.rn.f32x2", "max.f32", "max.f32 (3 inputs)", "max-plus mix")


def alu_probe(kind: int, iters: int = 4096, stream=None):
    """(instructions, element operations) per SM clock of one probe kind
    (`ALU_PROBE_KINDS`), measured by the library's register-only kernel."""
    lib = load_library()
    ins, elem = ctypes.c_double(), ctypes.c_double()
    rc = lib.esdp_alu_probe(kind, iters, ctypes.byref(ins), ctypes.byref(elem), _stream(stream))
    if rc != ESDP_OK:
        raise EsdpError(rc, "alu probe")
    return ins.value, elem.value
