"""The storage value J as a differentiable torch function.

    J(price, trans, eta_c, eta_d) = sum_k mu0[k] V_1[mode 0][s0][k]

Forward: one esdp_solve (backward induction, Algorithm 1 / eq. 5-6 on the
device) and esdp_objective.  Backward: esdp_grad, the hand-written adjoint: a
forward pass of the state-occupancy distribution under the stored argmax
policy (recomputed per segment from the V checkpoints when the asset keeps
checkpoints instead of the whole policy), which by the envelope theorem
gives dJ/dprice [T,K], dJ/dtrans [T,K,K] and dJ/deta_c, dJ/deta_d, exact
away from ties.  The per-action cost and the terminal value are data, held
fixed.

Torch supplies the device memory and the stream; every step of the solve
and of the adjoint runs in the CUDA library.
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import esdp as E


class StorageObjective:
    """J of one asset as a function of its prices, transition matrices and
    efficiencies.  `inst` fixes the shapes, the action band, s0, the policy
    storage (int32/int16, checkpoint interval), the cost, the terminal value
    and mu0.  Calling it returns a 0-dim float64 tensor that autograd can
    differentiate with respect to the tensors passed in."""

    def __init__(self, inst, device=None):
        self.template = copy.copy(inst)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        f32 = dict(dtype=torch.float32, device=self.device)
        self.cost = torch.as_tensor(np.ascontiguousarray(inst.cost), **f32)
        self.terminal = torch.as_tensor(np.ascontiguousarray(inst.terminal), **f32)
        self.mu0 = torch.as_tensor(np.ascontiguousarray(inst.mu0), **f32)
        self._solver = None
        self._eta = None
        self._solved = None   # token of the inputs of the context's last solve
        self._token = 0

    def solver(self, eta_c: float, eta_d: float) -> E.Solver:
        """The context for these efficiencies (action energies depend on them)."""
        if self._solver is None or self._eta != (eta_c, eta_d):
            if self._solver is not None:
                self._solver.close()
            inst = copy.copy(self.template)
            inst.eta_c, inst.eta_d = eta_c, eta_d
            with torch.cuda.device(self.device):
                self._solver = E.Solver([inst], device_ptrs=True)
            self._eta = (eta_c, eta_d)
            self._solved = None
        return self._solver

    def _solve(self, price, trans, eta_c, eta_d, token):
        s = self.solver(eta_c, eta_d)
        inst = self.template
        V1 = torch.empty(inst.n_modes * inst.N * inst.K, dtype=torch.float32, device=self.device)
        s.solve(price, trans, self.cost, self.terminal, V1)
        self._solved = token
        return s, V1

    def __call__(self, price, trans, eta_c=None, eta_d=None):
        T, K = self.template.T, self.template.K
        if tuple(price.shape) != (T, K) or tuple(trans.shape) != (T, K, K):
            raise ValueError(f"expected price [{T},{K}] and trans [{T},{K},{K}]")
        f64 = dict(dtype=torch.float64)
        eta_c = torch.tensor(self.template.eta_c, **f64) if eta_c is None else eta_c
        eta_d = torch.tensor(self.template.eta_d, **f64) if eta_d is None else eta_d
        return _Objective.apply(price, trans, eta_c, eta_d, self)


class _Objective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, price, trans, eta_c, eta_d, obj):
        p = price.detach().to(device=obj.device, dtype=torch.float32).contiguous()
        q = trans.detach().to(device=obj.device, dtype=torch.float32).contiguous()
        ec, ed = float(eta_c), float(eta_d)
        obj._token += 1
        token = obj._token
        s, _ = obj._solve(p, q, ec, ed, token)
        J = torch.empty(1, dtype=torch.float64, device=obj.device)
        s.objective(0, obj.mu0, J)
        ctx.obj, ctx.token, ctx.eta = obj, token, (ec, ed)
        ctx.meta = (price.dtype, price.device, trans.dtype, trans.device,
                    eta_c.dtype if torch.is_tensor(eta_c) else torch.float64,
                    eta_c.device if torch.is_tensor(eta_c) else torch.device("cpu"),
                    eta_d.dtype if torch.is_tensor(eta_d) else torch.float64,
                    eta_d.device if torch.is_tensor(eta_d) else torch.device("cpu"))
        ctx.save_for_backward(p, q)
        return J[0]

    @staticmethod
    def backward(ctx, gJ):
        obj = ctx.obj
        p, q = ctx.saved_tensors
        ec, ed = ctx.eta
        s = obj.solver(ec, ed)
        if obj._solved != ctx.token:
            # the context has solved other inputs since: recompute this solve
            s, _ = obj._solve(p, q, ec, ed, ctx.token)
        T, K = obj.template.T, obj.template.K
        dev = obj.device
        d_price = torch.empty((T, K), dtype=torch.float32, device=dev)
        d_trans = torch.empty((T, K, K), dtype=torch.float32, device=dev)
        d_eta = torch.empty(2, dtype=torch.float64, device=dev)
        s.grad(0, obj.mu0, None, d_price, d_trans, d_eta)
        g = gJ.to(dev)
        pdt, pdev, tdt, tdev, cdt, cdev, ddt, ddev = ctx.meta
        return ((g * d_price).to(pdev, pdt), (g * d_trans).to(tdev, tdt),
                (g * d_eta[0]).to(cdev, cdt), (g * d_eta[1]).to(ddev, ddt), None)
