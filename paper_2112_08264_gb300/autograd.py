"""Differentiable run: ``torch.autograd.Function`` over the library's adjoint.

Forward: a solver is created with coupling G, initialised at equilibrium
with zero velocity from (rho_A0, rho_B0), advanced ``nsteps`` steps while
recording checkpoints every ``ckpt_every`` steps; the final densities are
returned. Backward: ``lb_backward`` recomputes each checkpoint segment and
runs the hand-written adjoint step backwards through it, returning
dL/drho_A0, dL/drho_B0 and dL/dG. rho_A0 and rho_B0 are independent inputs;
for a tied rho_B0 = 1 - rho_A0 the gradient is dL/drho_A0 - dL/drho_B0.
"""
import torch

from .solver import Solver


class LBFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rhoA0, rhoB0, G, nsteps, ckpt_every, tau, mask, prec, kernel, body_force):
        nz, ny, nx = rhoA0.shape
        s = Solver(nx, ny, nz, tau, float(G.detach().cpu()), mask=mask, prec=prec, kernel=kernel,
                   body_force=body_force, ckpt_every=ckpt_every, ckpt_steps_max=nsteps, device=rhoA0.device)
        s.init(rhoA0.detach().float().contiguous(), rhoB0.detach().float().contiguous())
        s.step(nsteps)
        rA, rB, _ = s.moments(velocity=False)
        ctx.solver = s
        ctx.G_meta = (G.dtype, G.device)
        return rA, rB

    @staticmethod
    def backward(ctx, gA, gB):
        s = ctx.solver
        gA = gA.float().contiguous() if gA is not None else None
        gB = gB.float().contiguous() if gB is not None else None
        dA, dB, dG = s.backward(gA, gB)
        s.close()
        ctx.solver = None
        dtype, device = ctx.G_meta
        return dA, dB, torch.tensor(dG, dtype=dtype, device=device), None, None, None, None, None, None, None


def simulate(rhoA0, rhoB0, G, nsteps, ckpt_every=40, tau=1.0, mask=None, prec="fp32", kernel="fused",
             body_force=(0.0, 0.0, 0.0)):
    """Final (rho_A, rho_B) after ``nsteps``; differentiable in rho_A0, rho_B0
    and G (a 0-d tensor)."""
    if not isinstance(G, torch.Tensor):
        G = torch.tensor(float(G), dtype=torch.float64)
    return LBFunction.apply(rhoA0, rhoB0, G, int(nsteps), int(ckpt_every), float(tau), mask, prec, kernel,
                            tuple(body_force))
