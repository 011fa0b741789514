"""Gradients through SSP-RK3 time integration of the blended scheme.

`Evolve` is a torch.autograd.Function: u_T = Phi(u_0), n_steps SSP-RK3 steps of
the library's stage entry point. The blending coefficients of every stage and
every time step dt are those of the forward run and are held fixed in the
backward pass (the adjoint differentiates the scheme with the indicator's
output and the CFL step frozen). The backward pass is checkpointed: the
forward keeps the state every `every` steps and the time step of every step
(one float); the backward recomputes each segment from its checkpoint with
those time steps, recording the stage states and the coefficients the
indicator gives (the forward is deterministic, so they are the forward's own),
and runs the library's stage adjoint (sesc_rk_stage_vjp) stage by stage in
reverse. Device memory is then the checkpoints plus one segment's stage states
and coefficients, whatever the number of steps. With a plan given (frozen
coefficients per step), the plan is the caller's and is replayed.

All arithmetic runs in the library; this module only sequences the calls and
holds device buffers (torch tensors).
"""
import torch

RK3 = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))


def _step_record(solver, u, dt=None, coeffs=None):
    """One SSP-RK3 step from u. dt: None (CFL step computed) or a float;
    coeffs: None (indicator) or a list of three frozen coefficient tensors.
    Returns (u_new, record) with record = (dt, [us_1, us_2, us_3], [c_1, c_2, c_3])."""
    if dt is None:
        dt_dev = torch.empty(1, dtype=torch.float64, device=u.device)
        solver.dt(u, dt_dev)
        dt = float(dt_dev.item())
    stages, cs = [], []
    us = u
    for k, (a, b) in enumerate(RK3):
        c = torch.empty((solver.E, 2, solver.S), dtype=torch.float64, device=u.device)
        out = torch.empty_like(u)
        frozen = None if coeffs is None else coeffs[k]
        solver.rk_stage(u if a != 0.0 else None, us, out, a, b, dt=dt, frozen=frozen, coeffs_out=c)
        stages.append(us)
        cs.append(c if frozen is None else frozen)
        us = out
    return us, (dt, stages, cs)


def _step_vjp(solver, u, record, g):
    """Adjoint of one recorded step: returns dPhi/du^T g for u -> u_new."""
    dt, stages, cs = record
    u_bar = torch.zeros_like(u)
    gb = g
    for k in (2, 1, 0):
        a, b = RK3[k]
        us_bar = torch.empty_like(u)
        solver.rk_stage_vjp(stages[k], gb, us_bar, a, b, dt=dt, frozen=cs[k], u0_bar=u_bar)
        gb = us_bar
    # stage 1 has us = u: its us_bar is part of u_bar
    return u_bar + gb


def run(solver, u0, n_steps, plan=None):
    """Forward time loop; returns (u_T, plan) where plan lists (dt, coeffs) per step.
    With a plan given, the steps replay its dt and coefficients (frozen)."""
    u = u0
    out_plan = []
    for k in range(n_steps):
        dt, cf = (None, None) if plan is None else plan[k]
        u, rec = _step_record(solver, u, dt=dt, coeffs=cf)
        out_plan.append((rec[0], rec[2]))
    return u, out_plan


class Evolve(torch.autograd.Function):
    """u_T = Phi(u_0) with checkpointed adjoint (see module docstring)."""

    @staticmethod
    def forward(ctx, u0, solver, n_steps, every, plan, record):
        u = u0.detach()
        checkpoints = {0: u.clone()}
        dts = []
        for k in range(n_steps):
            dt, cf = (None, None) if plan is None else plan[k]
            u, rec = _step_record(solver, u, dt=dt, coeffs=cf)
            dts.append(rec[0])
            if record is not None:
                record.append((rec[0], rec[2]))
            if (k + 1) % every == 0 and k + 1 < n_steps:
                checkpoints[k + 1] = u.clone()
        ctx.solver, ctx.n_steps, ctx.every = solver, n_steps, every
        ctx.checkpoints = checkpoints
        ctx.dts = dts
        ctx.plan = plan
        return u

    @staticmethod
    def backward(ctx, g):
        solver = ctx.solver
        g = g.contiguous().to(torch.float64)
        starts = sorted(ctx.checkpoints)
        for s0 in reversed(starts):
            s1 = min(s0 + ctx.every, ctx.n_steps)
            # recompute the segment with the recorded dt / coefficients
            u = ctx.checkpoints[s0]
            records, states = [], []
            for k in range(s0, s1):
                cf = None if ctx.plan is None else ctx.plan[k][1]
                states.append(u)
                u, rec = _step_record(solver, u, dt=ctx.dts[k], coeffs=cf)
                records.append(rec)
            for k in range(s1 - s0 - 1, -1, -1):
                g = _step_vjp(solver, states[k], records[k], g)
        return g, None, None, None, None, None


def evolve(u0, solver, n_steps, every=20, plan=None, record=None):
    """Differentiable time loop (checkpoint every `every` steps). plan: replay the
    given (dt, coefficients) per step; record: a list that receives the plan used."""
    return Evolve.apply(u0, solver, n_steps, every, plan, record)
