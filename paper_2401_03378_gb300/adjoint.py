"""Gradients of a loss of the final state with respect to the initial fields.

The forward run advances nsteps SSP-RK2 steps with the CFL dt on the device,
keeping a copy of the state every `every` steps (checkpoints) and the dt of
every step.  The reverse sweep recomputes each segment from its checkpoint
stage by stage (hydro_stage with the recorded dt: the same launches as
hydro_step, so bitwise the forward states), keeping every step's state and
first-stage state, and applies hydro_step_adjoint_stored backwards.  dt is held fixed (its dependence on the
state is not differentiated) and every branch keeps its forward decision.
All arithmetic runs in libgbhydro's kernels; this module only schedules them.
"""
from __future__ import annotations

from typing import Dict, List

import torch

from .hydro import Hydro


class CheckpointedRun:
    def __init__(self, hydro: Hydro, nsteps: int, every: int = 10):
        if hydro.refined or hydro.nproblems != 1:
            raise ValueError("the adjoint runs on uniform single-problem contexts")
        self.h = hydro
        self.nsteps = int(nsteps)
        self.every = max(1, int(every))
        self.checkpoints: Dict[int, torch.Tensor] = {}
        self.dts: List[float] = []

    def forward(self, U0: torch.Tensor) -> torch.Tensor:
        U = U0.clone()
        dt = self.h.compute_dt(U)
        hist = torch.zeros(self.nsteps, dtype=torch.float64, device=U.device)
        self.checkpoints = {}
        for s in range(self.nsteps):
            if s % self.every == 0:
                self.checkpoints[s] = U.clone()
            self.h.advance(U, 1, dt, hist[s:s + 1])
        self.dts = [float(x) for x in hist.cpu()]
        return U

    def backward(self, lam_final: torch.Tensor) -> torch.Tensor:
        lam = lam_final.clone().contiguous()
        if self.h.nstages != 2 or self.h.telescoping:
            return self._backward_recompute(lam)
        for start in reversed(range(0, self.nsteps, self.every)):
            end = min(start + self.every, self.nsteps)
            states, firsts = [self.checkpoints[start].clone()], []
            for s in range(start, end):
                X, dt = states[-1], self.dts[s]
                U1 = torch.empty_like(X)
                self.h.stage(X, None, U1, dt, 0.0, 1.0)
                firsts.append(U1)
                if s < end - 1:
                    Xn = X.clone()
                    self.h.stage(U1, X, Xn, dt, 0.5, 0.5)
                    states.append(Xn)
            for s in reversed(range(start, end)):
                self.h.step_adjoint(states[s - start], self.dts[s], lam, lam, U1=firsts[s - start])
        return lam

    def _backward_recompute(self, lam: torch.Tensor) -> torch.Tensor:
        """Three-stage and telescoping contexts: the segment's states by
        hydro_step, each step's adjoint recomputing its intermediate stages."""
        for start in reversed(range(0, self.nsteps, self.every)):
            end = min(start + self.every, self.nsteps)
            states = [self.checkpoints[start].clone()]
            for s in range(start, end - 1):
                X = states[-1].clone()
                self.h.step(X, self.dts[s])
                states.append(X)
            for s in reversed(range(start, end)):
                self.h.step_adjoint(states[s - start], self.dts[s], lam, lam)
        return lam


class _Run(torch.autograd.Function):
    @staticmethod
    def forward(ctx, W0, hydro, nsteps, every):
        U0 = hydro.prim_to_cons(W0.contiguous())
        run = CheckpointedRun(hydro, nsteps, every)
        U = run.forward(U0)
        ctx.run = run
        ctx.hydro = hydro
        ctx.save_for_backward(W0)
        return U

    @staticmethod
    def backward(ctx, gU):
        (W0,) = ctx.saved_tensors
        lam0 = ctx.run.backward(gU.contiguous())
        gW = ctx.hydro.prim_to_cons_vjp(W0.contiguous(), lam0)
        return gW, None, None, None


def run_differentiable(hydro: Hydro, W0: torch.Tensor, nsteps: int, every: int = 10) -> torch.Tensor:
    """Final conserved state of nsteps steps from the primitive initial fields W0
    (state layout, variables rho, u, v, w, p), differentiable with respect to W0
    through the hand-written adjoint (checkpoint every `every` steps)."""
    return _Run.apply(W0, hydro, nsteps, every)
