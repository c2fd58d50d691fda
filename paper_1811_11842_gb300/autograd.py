"""torch.autograd.Function over N time steps (§4) with the hand-written
discrete adjoint of the library (`cahn_vjp`).

`phase_field_steps(phi0, chi, mobility, ...)` returns phi^N.  Its backward
gives the exact gradient of the discrete map with respect to phi0, chi and
M (up to the solver tolerance) by the adjoint time steps on the GPU, which
recompute the forward from checkpoints every `checkpoint` steps.  The
velocity and pressure start fields are inputs without gradient.  Any
objective built from phi^N in torch (for instance the detached-biofilm
volume, a weighted sum over the rows above a height) differentiates
through it.
"""
from __future__ import annotations

import torch

from . import binding, inputs


class PhaseFieldSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, chi, mobility, prm, u0, v0, p0, nsteps, checkpoint):
        q = prm.replace(chi=float(chi), mobility=float(mobility))
        start = [t.detach().to(torch.float64).clone() for t in (phi0, u0, v0, p0)]
        sim = binding.Simulation([q], [tuple(t.clone() for t in start)], device=phi0.device)
        try:
            sim.step(int(nsteps))
            phiN = sim.fields[0][0].clone()
        except Exception:
            sim.close()
            raise
        ctx.sim = sim
        ctx.start = start
        ctx.nsteps = int(nsteps)
        ctx.checkpoint = int(checkpoint)
        ctx.chi_dev = chi.device if torch.is_tensor(chi) else None
        ctx.mob_dev = mobility.device if torch.is_tensor(mobility) else None
        return phiN

    @staticmethod
    def backward(ctx, gphi):
        sim = ctx.sim
        try:
            phi0_bar, (chi_b, mob_b), _ = sim.vjp(0, *ctx.start, ctx.nsteps, ctx.checkpoint,
                                                  gphi.detach().to(torch.float64).contiguous())
        finally:
            sim.close()
        chi_g = (torch.tensor(chi_b, dtype=torch.float64, device=ctx.chi_dev)
                 if ctx.chi_dev is not None else None)
        mob_g = (torch.tensor(mob_b, dtype=torch.float64, device=ctx.mob_dev)
                 if ctx.mob_dev is not None else None)
        return phi0_bar, chi_g, mob_g, None, None, None, None, None, None


def phase_field_steps(phi0, chi, mobility, prm: "inputs.Params", u0, v0, p0, nsteps: int,
                      checkpoint: int = 10):
    """phi^N after nsteps steps from a fresh start; differentiable in phi0,
    chi and mobility (0-dim tensors with requires_grad, or floats)."""
    return PhaseFieldSteps.apply(phi0, chi, mobility, prm, u0, v0, p0, nsteps, checkpoint)


def detached_volume_weights(prm: "inputs.Params", y_cut: float = 0.25, device="cuda:0"):
    """Weights of J = sum over rows with y_j > y_cut of w_ij phi_ij hx hy
    (trapezoid w, 1/2 on the wall rows; rows exactly at y_cut excluded)."""
    hx, hy = prm.lx / prm.nx, prm.ly / prm.ny
    y = torch.arange(prm.ny + 1, dtype=torch.float64) * hy
    w = torch.ones(prm.ny + 1, dtype=torch.float64)
    w[0] = w[-1] = 0.5
    rows = (y > y_cut).to(torch.float64) * w * hx * hy
    return rows[:, None].expand(prm.ny + 1, prm.nx).contiguous().to(device)
