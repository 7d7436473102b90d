"""torch.autograd wrapper of the IPC step and its implicit adjoint.

`IpcStep.apply(sim, step, logE, mu, z_t, zd_t)` advances one step on the GPU
(sim_step) and returns (z_{t+1}, zd_{t+1}); its backward calls sim_adjoint,
which recomputes the step's Hessian at the converged positions from the
saved checkpoint (z_t, zd_t, z_{t+1}) and the step's joint drive targets and
solves the adjoint system.  The
parameters are the per-tet ln Young's modulus and the friction coefficient
(material and friction identification from trajectories).
"""
from __future__ import annotations

import torch


class IpcStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sim, step, logE, mu, z_t, zd_t):
        sim.set_params(logE.detach().cpu().numpy(), float(mu))
        sim.set_dofs(z_t.detach(), zd_t.detach())
        T = sim.scene["kin_T"]
        if sim.nkb:
            sim.set_kinematic(T[step])
        jt = sim.joint_targets(step + 1)
        sim.step(T[step + 1] if sim.nkb else None, joint_targets=jt if jt[0] is not None else None)
        z_next, zd_next = sim.get_dofs()
        ctx.sim = sim
        ctx.step = step
        ctx.logE = logE.detach().cpu().numpy()
        ctx.mu = float(mu)
        ctx.save_for_backward(z_t.detach(), zd_t.detach(), z_next)
        return z_next, zd_next

    @staticmethod
    def backward(ctx, gz, gzd):
        sim = ctx.sim
        z_t, zd_t, z_next = ctx.saved_tensors
        sim.set_params(ctx.logE, ctx.mu)
        if gz is None:
            gz = torch.zeros_like(z_next)
        if gzd is None:
            gzd = torch.zeros_like(z_next)
        T = sim.scene["kin_T"]
        gz_t, gzd_t, glogE, gmu = sim.adjoint(z_t, zd_t, z_next, T[ctx.step] if sim.nkb else None,
                                              T[ctx.step + 1] if sim.nkb else None, gz.double(), gzd.double(),
                                              step_next=ctx.step + 1)
        dev = ctx.needs_input_grad
        return (None, None, glogE.to("cpu") if dev[2] else None,
                torch.tensor(gmu, dtype=torch.float64) if dev[3] else None, gz_t, gzd_t)


def rollout(sim, logE, mu, n_steps, z0=None, zd0=None):
    """Differentiable rollout of n_steps from (z0, zd0) (default: the simulator's current state)."""
    if z0 is None:
        z0, zd0 = sim.get_dofs()
    z, zd = z0, zd0
    traj = []
    for k in range(n_steps):
        z, zd = IpcStep.apply(sim, k, logE, mu, z, zd)
        traj.append(z)
    return traj
