"""The storage value J as a differentiable torch function.

    J(price, trans, eta_c, eta_d, switch_cost, cost, terminal, mu0)
        = sum_k mu0[k] V_1[mode 0][s0][k]

Forward: one esdp_solve (backward induction, Algorithm 1 / eq. 5-6 on the
device) and esdp_objective.  Backward: esdp_grad, the hand-written adjoint: a
forward pass of the state-occupancy distribution under the stored argmax
policy (recomputed per segment from the V checkpoints when the asset keeps
checkpoints instead of the whole policy), which by the envelope theorem
gives every sensitivity at once, exact away from ties:
dJ/dprice [T,K], dJ/dtrans [T,K,K], dJ/deta_c, dJ/deta_d, dJ/dswitch_cost,
dJ/dcost [A], dJ/dterminal [n_modes,N,K] (the final occupancy) and
dJ/dmu0 [K] (= V_1[0][s0][:]).

Torch supplies the device memory and the stream; every step of the solve
and of the adjoint runs in the CUDA library.
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import esdp as E


class StorageObjective:
    """J of one asset.  `inst` fixes the shapes, the action band, s0 and the
    policy storage (int32/int16, checkpoint interval) and gives the default
    values of every input.  Calling it returns a 0-dim float64 tensor that
    autograd can differentiate with respect to the tensors passed in."""

    def __init__(self, inst, device=None):
        self.template = copy.copy(inst)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        f32 = dict(dtype=torch.float32, device=self.device)
        self.cost = torch.as_tensor(np.ascontiguousarray(inst.cost), **f32)
        self.terminal = torch.as_tensor(np.ascontiguousarray(inst.terminal), **f32)
        self.mu0 = torch.as_tensor(np.ascontiguousarray(inst.mu0), **f32)
        self._solver = None
        self._scalars = None
        self._solved = None   # token of the inputs of the context's last solve
        self._token = 0

    def solver(self, eta_c: float, eta_d: float, switch_cost: float) -> E.Solver:
        """The context for these scalars (action energies and the mode
        payoffs depend on them)."""
        key = (eta_c, eta_d, switch_cost)
        if self._solver is None or self._scalars != key:
            if self._solver is not None:
                self._solver.close()
            inst = copy.copy(self.template)
            inst.eta_c, inst.eta_d, inst.switch_cost = key
            with torch.cuda.device(self.device):
                self._solver = E.Solver([inst], device_ptrs=True)
            self._scalars = key
            self._solved = None
        return self._solver

    def _solve(self, args, token):
        price, trans, cost, terminal = args["price"], args["trans"], args["cost"], args["terminal"]
        s = self.solver(*args["scalars"])
        inst = self.template
        V1 = torch.empty(inst.n_modes * inst.N * inst.K, dtype=torch.float32, device=self.device)
        s.solve(price, trans, cost, terminal, V1)
        self._solved = token
        return s

    def __call__(self, price, trans, eta_c=None, eta_d=None, switch_cost=None, cost=None,
                 terminal=None, mu0=None):
        inst = self.template
        T, K = inst.T, inst.K
        if tuple(price.shape) != (T, K) or tuple(trans.shape) != (T, K, K):
            raise ValueError(f"expected price [{T},{K}] and trans [{T},{K},{K}]")
        f64 = dict(dtype=torch.float64)
        eta_c = torch.tensor(inst.eta_c, **f64) if eta_c is None else eta_c
        eta_d = torch.tensor(inst.eta_d, **f64) if eta_d is None else eta_d
        switch_cost = torch.tensor(inst.switch_cost, **f64) if switch_cost is None else switch_cost
        cost = self.cost if cost is None else cost
        terminal = self.terminal if terminal is None else terminal
        mu0 = self.mu0 if mu0 is None else mu0
        if tuple(cost.shape) != (inst.A,) or tuple(terminal.shape) != (inst.n_modes, inst.N, K) \
                or tuple(mu0.shape) != (K,):
            raise ValueError("cost [A], terminal [n_modes,N,K] and mu0 [K] expected")
        return _Objective.apply(price, trans, eta_c, eta_d, switch_cost, cost, terminal, mu0, self)


def _dev(x, obj):
    return x.detach().to(device=obj.device, dtype=torch.float32).contiguous()


class _Objective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, price, trans, eta_c, eta_d, switch_cost, cost, terminal, mu0, obj):
        args = {"price": _dev(price, obj), "trans": _dev(trans, obj), "cost": _dev(cost, obj),
                "terminal": _dev(terminal, obj), "mu0": _dev(mu0, obj),
                "scalars": (float(eta_c), float(eta_d), float(switch_cost))}
        obj._token += 1
        token = obj._token
        s = obj._solve(args, token)
        J = torch.empty(1, dtype=torch.float64, device=obj.device)
        s.objective(0, args["mu0"], J)
        ctx.obj, ctx.token, ctx.args = obj, token, args
        ctx.like = [(x.dtype, x.device) if torch.is_tensor(x) else (torch.float64, torch.device("cpu"))
                    for x in (price, trans, eta_c, eta_d, switch_cost, cost, terminal, mu0)]
        return J[0]

    @staticmethod
    def backward(ctx, gJ):
        obj, args = ctx.obj, ctx.args
        s = obj.solver(*args["scalars"])
        if obj._solved != ctx.token:
            # the context has solved other inputs since: recompute this solve
            s = obj._solve(args, ctx.token)
        inst = obj.template
        T, K, dev = inst.T, inst.K, obj.device
        f32 = dict(dtype=torch.float32, device=dev)
        d_price = torch.empty((T, K), **f32)
        d_trans = torch.empty((T, K, K), **f32)
        d_eta = torch.empty(2, dtype=torch.float64, device=dev)
        d_cost = torch.empty(inst.A, **f32)
        d_sw = torch.empty(1, dtype=torch.float64, device=dev)
        d_term = torch.empty((inst.n_modes, inst.N, K), **f32)
        d_mu0 = torch.empty(K, **f32)
        s.grad(0, args["mu0"], None, d_price, d_trans, d_eta, d_cost, d_sw, d_term, d_mu0)
        g = gJ.to(dev)
        grads = (d_price, d_trans, d_eta[0], d_eta[1], d_sw[0], d_cost, d_term, d_mu0)
        return tuple((g * d).to(dev_, dt) for d, (dt, dev_) in zip(grads, ctx.like)) + (None,)
