"""torch.autograd binding of the rigid-pose energy (the derivative of Eq. EnergySum_ligand
with respect to translation and rotation vector).

The forward pass runs the adjoint kernel once (rs_energy_grad_poses), which returns
E together with dE/dt and dE/dw; backward only scales those by the incoming
gradient.  Nothing is computed in Python.
"""
from __future__ import annotations

import torch

from . import lib


class RSEnergy(torch.autograd.Function):
    """E(rotvec, trans) for a batch of rigid poses; differentiable in rotvec and trans."""

    @staticmethod
    def forward(fctx, rotvec, trans, ctx_handle, prot_handle, lig_xyz, lig_q):
        E, gt, gw, flags = lib.rs_energy_grad_poses(ctx_handle, prot_handle, lig_xyz, lig_q,
                                                    rotvec.detach().contiguous(),
                                                    trans.detach().contiguous())
        fctx.save_for_backward(gt, gw)
        fctx.mark_non_differentiable(flags)
        return E, flags

    @staticmethod
    def backward(fctx, gE, gflags):
        gt, gw = fctx.saved_tensors
        g = gE.to(gt.dtype)[:, None]
        return g * gw, g * gt, None, None, None, None


def rs_energy(protein: "lib.Protein", lig_xyz, lig_q, rotvec, trans):
    """Differentiable energies (and non-differentiable vdW flags) of poses given by
    rotation vectors and translations (CUDA float64 tensors [P, 3])."""
    return RSEnergy.apply(rotvec, trans, protein.ctx.handle, protein.handle, lig_xyz, lig_q)
