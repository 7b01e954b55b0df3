"""torch.autograd binding of the library's misfit gradient (loss_gradient): the seismogram misfit of one shot
as a differentiable function of the vp / vs / rho grids.

    J = seismogram_misfit(vp, vs, rho, grid, shot, d_obs, n_steps)
    J.backward()          # vp.grad, vs.grad, rho.grad from the hand-written discrete adjoint

The forward call runs the library's forward and adjoint passes together (checkpointed recomputation of the
wavefield on the GPU); backward only scales the stored gradients.  Argument marshalling only.
"""
from __future__ import annotations

import torch


class SeismogramMisfit(torch.autograd.Function):
    """J(vp, vs, rho) = 1/2 sum (traces - d_obs)^2 over n_steps steps of shot ``shot`` of ``grid`` from rest."""

    @staticmethod
    def forward(ctx, vp, vs, rho, grid, shot, d_obs, n_steps, checkpoint_every=0):
        grid.set_model(shot, vp, vs, rho)
        J, g = grid.gradient(shot, d_obs, n_steps, checkpoint_every)
        dev = vp.device
        gvp = g["vp"].to(dev) if isinstance(g["vp"], torch.Tensor) else torch.from_numpy(g["vp"]).to(dev)
        grho = g["rho"].to(dev) if isinstance(g["rho"], torch.Tensor) else torch.from_numpy(g["rho"]).to(dev)
        if vs is not None:
            gvs = g["vs"].to(dev) if isinstance(g["vs"], torch.Tensor) else torch.from_numpy(g["vs"]).to(dev)
        else:
            gvs = torch.zeros(0, dtype=torch.float64, device=dev)
        ctx.has_vs = vs is not None
        ctx.save_for_backward(gvp.to(vp.dtype), gvs, grho.to(rho.dtype))
        return torch.tensor(J, dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, gJ):
        gvp, gvs, grho = ctx.saved_tensors
        return gJ * gvp, (gJ * gvs if ctx.has_vs else None), gJ * grho, None, None, None, None, None


def seismogram_misfit(vp, vs, rho, grid, shot, d_obs, n_steps, checkpoint_every=0):
    """Differentiable misfit; see SeismogramMisfit.  vs is None for acoustic grids."""
    return SeismogramMisfit.apply(vp, vs, rho, grid, shot, d_obs, n_steps, checkpoint_every)
