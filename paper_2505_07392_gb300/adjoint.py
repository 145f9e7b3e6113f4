"""Gradients through many SSP-RK3 steps with the hand-written adjoint.

The objective of the jet workload is the time-integrated mean pressure on a
horizontal plane,
    J(w) = sum_{n=1..N} dt * mean_{i,j} (p(q^n)_{k} + p(q^n)_{k+1}) / 2,
where the plane lies on the face between cell layers k and k+1 and w are the
jets' inflow velocities. dJ/dw comes from the reverse sweep
    lambda_N = dt dP/dq^N,
    (lambda_{n-1}, mu_{n-1}, g) = adjoint of step n-1 -> n applied to (lambda_n, mu_n),
    lambda_{n-1} += dt dP/dq^{n-1},
with every step's adjoint computed by igr_adjoint_step (kernels only). The
forward keeps a checkpoint (q, Sigma) every `checkpoint_every` steps and each
segment is recomputed during the reverse sweep, so memory holds one segment.
The pressure objective and its derivative dP/dq are the caller's objective,
evaluated with torch on the device.

IGRStep and JetRollout expose the two as torch.autograd.Functions.
"""
from __future__ import annotations

from dataclasses import replace

import torch

from . import igr


def plane_pressure(q: torch.Tensor, k: int, gamma: float) -> torch.Tensor:
    """mean_{i,j} (p_k + p_{k+1}) / 2 of a (5, nz, ny, nx) state."""
    q = q[:, k:k + 2]
    rho, mx, my, mz, E = q[0], q[1], q[2], q[3], q[4]
    p = (gamma - 1.0) * (E - 0.5 * (mx * mx + my * my + mz * mz) / rho)
    return p.mean()


def _dP(q: torch.Tensor, k: int, gamma: float) -> torch.Tensor:
    # grad mode is off inside an autograd.Function's forward
    with torch.enable_grad():
        x = q.detach().to(torch.float64).requires_grad_(True)
        (g,) = torch.autograd.grad(plane_pressure(x, k, gamma), x)
    return g


def with_jet_velocities(case, w):
    jets = [tuple(j[:4]) + (float(wj),) + tuple(j[5:]) for j, wj in zip(case.jets, w)]
    return replace(case, jets=jets)


def rollout_jet_gradient(case, precision, q0, nsteps, dt, plane_k, checkpoint_every=30,
                         sigma0=None):
    """(J, dJ/dw) for the plane-pressure objective; q0 is a device tensor."""
    ct = torch.float64 if precision == "f64" else torch.float32
    with igr.Solver(case, precision) as s:
        st = igr.storage_torch_dtype(precision)
        s.set_state(q0.to(st), None if sigma0 is None else sigma0.to(st))
        ckpt = {0: s.get_state()}
        J = 0.0
        for n in range(1, nsteps + 1):
            s.step(1, fixed_dt=dt, sync=False)
            q, sig = s.get_state()
            J += dt * float(plane_pressure(q.to(torch.float64), plane_k, case.gamma))
            if n % checkpoint_every == 0 and n < nsteps:
                ckpt[n] = (q, sig)
        # reverse sweep, one recomputed segment at a time
        lam_q = torch.zeros((5,) + s.shape, dtype=ct, device=s.device)
        lam_s = torch.zeros(s.shape, dtype=ct, device=s.device)
        gw = [0.0] * len(case.jets)
        starts = sorted(ckpt)
        for seg, m in reversed(list(enumerate(starts))):
            end = starts[seg + 1] if seg + 1 < len(starts) else nsteps
            s.set_state(*ckpt[m])
            states = [ckpt[m]]
            for _ in range(m, end):
                s.step(1, fixed_dt=dt, sync=False)
                states.append(s.get_state())
            for n in range(end, m, -1):
                qn, _ = states[n - m]
                lam_q = lam_q + (dt * _dP(qn, plane_k, case.gamma)).to(ct)
                qp, sp = states[n - 1 - m]
                lam_q, lam_s, g = s.adjoint_step(qp, sp, lam_q, lam_s, dt)
                gw = [a + b for a, b in zip(gw, g)]
        return J, gw


class IGRStep(torch.autograd.Function):
    """One SSP-RK3 step with fixed dt as a differentiable torch op:
    (q, Sigma) -> (q', Sigma') on a Solver; backward runs igr_adjoint_step."""

    @staticmethod
    def forward(ctx, q, sigma, solver, dt):
        st = igr.storage_torch_dtype(solver.precision)
        qs, ss = q.detach().to(st).contiguous(), sigma.detach().to(st).contiguous()
        solver.set_state(qs, ss)
        solver.step(1, fixed_dt=dt, sync=False)
        q1, s1 = solver.get_state(igr.compute_torch_dtype(solver.precision))
        ctx.solver, ctx.dt = solver, dt
        ctx.save_for_backward(qs, ss)
        return q1, s1

    @staticmethod
    def backward(ctx, gq, gs):
        qs, ss = ctx.saved_tensors
        if gq is None:
            gq = torch.zeros((5,) + ctx.solver.shape, dtype=igr.compute_torch_dtype(ctx.solver.precision),
                             device=qs.device)
        if gs is None:
            gs = torch.zeros(ctx.solver.shape, dtype=gq.dtype, device=qs.device)
        lq, ls, _ = ctx.solver.adjoint_step(qs, ss, gq, gs, ctx.dt)
        return lq, ls, None, None


class JetRollout(torch.autograd.Function):
    """J(w) of `rollout_jet_gradient` as a differentiable function of the jet
    velocities w (a 1-D CPU tensor); the forward computes the gradient by the
    checkpointed adjoint and backward returns it."""

    @staticmethod
    def forward(ctx, w, case, precision, q0, nsteps, dt, plane_k, checkpoint_every):
        c = with_jet_velocities(case, w.tolist())
        J, gw = rollout_jet_gradient(c, precision, q0, nsteps, dt, plane_k, checkpoint_every)
        ctx.save_for_backward(torch.tensor(gw, dtype=torch.float64))
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        (gw,) = ctx.saved_tensors
        return (gJ * gw).to(torch.float64), None, None, None, None, None, None, None
