"""Energy of charges plus induced point dipoles as a differentiable function.

Forward: build the octree, run the static pass and solve the induced dipoles
(Sec. III, stages 1 and 2); the library reduces the energy in the stationary
form U^pol = -1/2 sum mu.E^q, valid at the solution (Eq. upol_derivatives).
Backward: one more FMM pass with charges and dipoles as sources (stage 3).
Because dU^pol/dmu = 0 at the solution, the gradients need no derivative of
the dipole iterations: dU/dx = -(q E + (grad E) mu), dU/dq = Phi,
dU/dalpha = -|mu|^2 / (2 alpha^2).
"""
from __future__ import annotations

import torch


class _PolarizableEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, q, alpha, p, depth, mode, tol, max_iter, coulomb_k, root_box):
        from . import PolFMM

        fmm = PolFMM(pos.detach(), q.detach(), alpha.detach(), p=p, depth=depth, mode=mode, max_iter=max_iter,
                     coulomb_k=coulomb_k, root_box=root_box)
        info = fmm.solve(tol)
        out = fmm.energy_forces(forces=True, dq=True, dalpha=True)
        ctx.info = info
        ctx.grads = (-out["F"], out["dUdq"], out["dUdalpha"])
        fmm.close()
        return torch.tensor(out["U"], dtype=torch.float64, device=pos.device)

    @staticmethod
    def backward(ctx, gU):
        gx, gq, ga = ctx.grads
        return gU * gx, gU * gq, gU * ga, None, None, None, None, None, None, None


class _PolarizableEnergyTwoPass(torch.autograd.Function):
    """Forward keeps the context (tree, static pass, dipoles) and takes the
    stationary energy from the library; the first backward runs the force pass
    on it, so the gradient pass happens only when asked for.  The gradients are
    kept, so a second backward (retain_graph=True) reuses them."""

    @staticmethod
    def forward(ctx, pos, q, alpha, p, depth, mode, tol, max_iter, coulomb_k, root_box):
        from . import PolFMM

        fmm = PolFMM(pos.detach(), q.detach(), alpha.detach(), p=p, depth=depth, mode=mode, max_iter=max_iter,
                     coulomb_k=coulomb_k, root_box=root_box)
        info = fmm.solve(tol)
        U = fmm.energy()["U"]
        ctx.fmm = fmm
        ctx.info = info
        ctx.grads = None
        return torch.tensor(U, dtype=torch.float64, device=pos.device)

    @staticmethod
    def backward(ctx, gU):
        if ctx.grads is None:
            out = ctx.fmm.energy_forces(forces=True, dq=True, dalpha=True)
            ctx.fmm.close()
            ctx.fmm = None
            ctx.grads = (-out["F"], out["dUdq"], out["dUdalpha"])
        gx, gq, ga = ctx.grads
        return gU * gx, gU * gq, gU * ga, None, None, None, None, None, None, None


def polarizable_energy(pos, q, alpha, p=6, depth=4, mode="fp64", tol=1e-8, max_iter=200, coulomb_k=1.0,
                       keep_context=True, root_box=None):
    """U(pos, q, alpha) for CUDA float64 tensors; differentiable in all three.

    keep_context=True keeps the tree, static pass and dipoles from the forward
    pass and runs the force pass in backward; False computes the gradients in
    forward and frees the device state at once.  root_box = (lo[3], side)
    fixes the root cube (e.g. for finite differences, so that no site changes
    leaf); None uses the bounding cube of the positions."""
    if keep_context:
        return _PolarizableEnergyTwoPass.apply(pos, q, alpha, p, depth, mode, tol, max_iter, coulomb_k, root_box)
    return _PolarizableEnergy.apply(pos, q, alpha, p, depth, mode, tol, max_iter, coulomb_k, root_box)
