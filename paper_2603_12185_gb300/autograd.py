"""Differentiable rollouts: a torch.autograd.Function over cf_step / cf_step_grad.

forward:  (q0, v0, tau[T, total_nu]) -> (q_T, v_T), T steps of the batched ComFree step.
backward: the library's adjoint (checkpointed recomputation of the trajectory, exact per-step
          vector-Jacobian products) maps (dL/dq_T, dL/dv_T) to (dL/dq0, dL/dv0, dL/dtau).
"""
from __future__ import annotations

import torch


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, batch, dt, q0, v0, tau):
        T = tau.shape[0]
        batch.set_state(q0.detach(), v0.detach())
        batch.set_ctrl(tau.detach().reshape(-1))
        batch.step(dt, T)
        qT, vT = batch.get_state()
        ctx.batch, ctx.dt, ctx.T = batch, dt, T
        ctx.save_for_backward(q0.detach().clone(), v0.detach().clone(), tau.detach().clone())
        return qT, vT

    @staticmethod
    def backward(ctx, gq, gv):
        q0, v0, tau = ctx.saved_tensors
        b = ctx.batch
        gq = torch.zeros(b.total_nq, device=q0.device) if gq is None else gq.float()
        gv = torch.zeros(b.total_nv, device=q0.device) if gv is None else gv.float()
        b.set_state(q0, v0)
        b.set_ctrl(tau.reshape(-1))
        dq0, dv0, dtau = b.step_grad(ctx.T, ctx.dt, gq, gv)
        return None, None, dq0, dv0, dtau.reshape(tau.shape)


def rollout(batch, dt, q0, v0, tau):
    """Differentiable T-step rollout; tau is [T, total_nu] (actuated hinge torques)."""
    return Rollout.apply(batch, dt, q0, v0, tau)
