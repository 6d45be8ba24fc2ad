"""Differentiable simulation: rho_T, u_T = LBMFunction.apply(sim, T, K, f0, force).

Forward: T steps of the library from the canonical state f0 (or the context's
current state when f0 is None), with the per-node body force `force` (or the
context's uniform force when None); a native checkpoint of the lattice is
kept every K steps (K ~ sqrt(T) balances memory and recompute), plus the
final state.

Backward (hand-written discrete adjoint, all in the library's kernels):
  1. lbm_macros_backward at A_T turns dL/drho_T, dL/du_T into lambda_T =
     dL/dA_T and starts dL/dF;
  2. for each segment, last first: lbm_forward_states recomputes the
     segment's states from its checkpoint into reused buffers, and
     lbm_backward runs the adjoint steps back through them, accumulating
     dL/dF.
Gradients are returned for f0 (dL/dA_0, canonical [9, ny, nx]) and for the
per-node force field ([2, ny, nx]); the gradient of a uniform force is the
node sum of the latter.

The context's lattice holds A_T after the forward and again after the
backward (the backward reloads the saved final state).
"""
from __future__ import annotations

import math
from typing import List, Optional, Tuple

import torch

from .lbm import LBM


def checkpoint_segments(T: int, K: int) -> List[Tuple[int, int]]:
    """(start step, steps) of each checkpoint segment covering [0, T)."""
    if T < 0 or K < 1:
        raise ValueError("need T >= 0 and K >= 1")
    return [(s, min(K, T - s)) for s in range(0, T, K)]


def default_interval(T: int) -> int:
    """Checkpoint interval ~ sqrt(T) (45 for T = 2000)."""
    return max(1, int(round(math.sqrt(max(T, 1)))))


class LBMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sim: LBM, T: int, K: int, f0: Optional[torch.Tensor], force: Optional[torch.Tensor]):
        if f0 is not None:
            sim.set_f(f0.detach())
        sim.set_force(None if force is None else force.detach())
        segs = checkpoint_segments(T, K)
        t_start = sim.steps
        ckpts = []
        for (_, n) in segs:
            ckpts.append(sim.save_state())
            sim.step(n)
        final = sim.save_state()
        rho, u = sim.macros()
        ctx.sim, ctx.T, ctx.K = sim, T, K
        ctx.ckpts, ctx.final, ctx.segs, ctx.t_start = ckpts, final, segs, t_start
        ctx.has_f0, ctx.has_force = f0 is not None, force is not None
        return rho, u

    @staticmethod
    def backward(ctx, g_rho, g_u):
        sim: LBM = ctx.sim
        ny, nx, dt = sim.ny, sim.nx, sim.dtype
        dev = sim.device
        lam = torch.empty((9, ny, nx), dtype=dt, device=dev)
        lam_tmp = torch.empty_like(lam)
        gF = torch.zeros((2, ny, nx), dtype=dt, device=dev)
        sim.load_state(ctx.final)
        sim.macros_backward(None if g_rho is None else g_rho.contiguous(),
                            None if g_u is None else g_u.contiguous(), lam, gF)
        # every segment runs on the same K state buffers (the checkpoint is
        # copied into the first), so that the recompute and the adjoint sweep
        # of all full segments replay one recorded CUDA graph each
        bufs = [sim.new_state() for _ in range(max(1, ctx.K))]
        for s in range(len(ctx.segs) - 1, -1, -1):
            start, n = ctx.segs[s]
            bufs[0].copy_(ctx.ckpts[s])
            states = bufs[:n]
            if n > 1:
                sim.forward_states(states, ctx.t_start + start)
            sim.backward(states, lam, lam_tmp, gF)
        sim.load_state(ctx.final)
        return (None, None, None, lam if ctx.has_f0 else None, gF if ctx.has_force else None)


def simulate(sim: LBM, T: int, f0: Optional[torch.Tensor] = None, force: Optional[torch.Tensor] = None,
             K: Optional[int] = None):
    """(rho_T, u_T), differentiable w.r.t. f0 and force."""
    return LBMFunction.apply(sim, int(T), int(K or default_interval(T)), f0, force)
