"""Gradient of the time-integrated right-edge leakage with respect to per-cell
opacity scales, as a ``torch.autograd.Function`` over the library's forward
steps (``sm_ho_step``) and adjoint steps (``sm_adjoint_step``).

Memory is bounded by time-step checkpointing: the forward keeps the
temperature of every step (one nodal array each) but the intensity only at
every ``checkpoint_every``-th step; the backward recomputes one segment at a
time from its checkpoint and runs the adjoint steps of that segment in
reverse.  Packed intensities held at once: (number of checkpoints) + (one
segment) + 2 adjoint buffers.

Argument marshalling only: every step runs in the library's CUDA kernels.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import torch

from . import Problem


def equilibrium_intensity(prob: Problem, T):
    """Packed intensity B_g(T)/4pi at every node and direction (the emission
    with unit opacity), for an equilibrium initial state."""
    i = prob.info
    ones = torch.ones((i["n_groups"], i["n_cells"]), dtype=torch.float64, device="cuda")
    b = prob.emission(T, ones)
    canon = b.unsqueeze(0).expand(i["n_dir"], -1, -1, -1).contiguous()
    return prob.pack(canon)


@dataclasses.dataclass
class LeakageSetup:
    """What the objective needs besides the opacity scales."""
    prob: Problem
    cv: torch.Tensor          # [cell][node]
    T0: torch.Tensor          # [cell][node]
    I0: torch.Tensor          # packed initial intensity
    nsteps: int
    checkpoint_every: int = 0  # 0: sqrt(nsteps)
    tol: float = 1e-13
    max_iter: int = 1000
    dt: float = 0.0            # the problem's time step (for the objective's quadrature)

    def every(self) -> int:
        if self.checkpoint_every > 0:
            return self.checkpoint_every
        return max(1, int(round(math.sqrt(self.nsteps))))


class _Leakage(torch.autograd.Function):
    @staticmethod
    def forward(ctx, scale, setup: LeakageSetup):
        prob = setup.prob
        k = setup.every()
        T = setup.T0.clone()
        I_cur = setup.I0
        Ts: List[torch.Tensor] = [T.clone()]
        ckpt = {0: setup.I0.clone()}
        J = 0.0
        iters = []
        for n in range(setup.nsteps):
            I_next = prob.empty_intensity()
            iters.append(prob.ho_step(scale, setup.cv, T, I_cur, I_next, setup.tol,
                                      setup.max_iter))
            J += setup.dt * prob.leakage(I_next)
            Ts.append(T.clone())
            if (n + 1) % k == 0 and n + 1 < setup.nsteps:
                ckpt[n + 1] = I_next
            I_cur = I_next
        ctx.setup = setup
        ctx.Ts = Ts
        ctx.ckpt = ckpt
        ctx.forward_iters = iters
        ctx.save_for_backward(scale)
        return torch.tensor(J, dtype=torch.float64, device=scale.device)

    @staticmethod
    def backward(ctx, gJ):
        (scale,) = ctx.saved_tensors
        setup = ctx.setup
        prob = setup.prob
        k = setup.every()
        N = setup.nsteps
        grad = torch.zeros_like(scale)
        psi = [prob.empty_intensity(), prob.empty_intensity()]
        X = [torch.zeros_like(setup.T0), torch.zeros_like(setup.T0)]
        have_next = False
        cur = 0
        adj_iters = []
        for start in range(((N - 1) // k) * k, -1, -k):
            end = min(start + k, N)
            # recompute the segment's intensities from its checkpoint
            T = ctx.Ts[start].clone()
            Is = {start: ctx.ckpt[start]}
            for n in range(start, end):
                Is[n + 1] = prob.empty_intensity()
                prob.ho_step(scale, setup.cv, T, Is[n], Is[n + 1], setup.tol, setup.max_iter)
            for n in range(end - 1, start - 1, -1):
                nxt = 1 - cur
                adj_iters.append(prob.adjoint_step(
                    scale, setup.cv, ctx.Ts[n], ctx.Ts[n + 1], Is[n + 1],
                    psi[cur] if have_next else None, X[cur] if have_next else None,
                    psi[nxt], X[nxt], grad, setup.tol, setup.max_iter))
                cur = nxt
                have_next = True
            del Is
        ctx.adjoint_iters = adj_iters[::-1]
        return gJ * grad, None


def leakage(scale: torch.Tensor, setup: LeakageSetup) -> torch.Tensor:
    """J(s) = sum_n dt * (right-edge outgoing partial current of I^{n+1}),
    differentiable in the per-cell opacity scales s (FP64, on the device)."""
    return _Leakage.apply(scale, setup)
