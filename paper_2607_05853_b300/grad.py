"""Differentiable lowest exciton energies: a torch.autograd.Function whose forward runs the
library's assembly and Lanczos, and whose backward is the library's hand-written adjoint.

    Omega = ExcitonEnergies.apply(W_R, e_qp, bse, fixed, n_eig, n_steps, seed)

W_R ([n_RW][N_aux][N_aux] float64) and e_qp ([N_k][nv+nc] float64) are the differentiable
inputs; `fixed` holds the device tensors V0, C_R, c_k of the same crystal.  The backward
builds the Hellmann-Feynman seed sum_s g_s x_s x_s^dagger from the Ritz vectors of the forward
(bse_adjoint_seed) and contracts it through the assembly (bse_adjoint), recomputing the pair
projections instead of storing them.  Only the binding's calls run; no arithmetic here.
"""
from __future__ import annotations

import torch

from .api import BSE

__all__ = ["ExcitonEnergies"]


class ExcitonEnergies(torch.autograd.Function):
    @staticmethod
    def forward(ctx, W_R: torch.Tensor, e_qp: torch.Tensor, bse: BSE, fixed: dict, n_eig: int, n_steps: int,
                seed: int = 12345):
        bse.interp_W(W_R.detach().contiguous(), fixed["V0"])
        bse.project_pairs(fixed["C_R"], fixed["c_k"], e_qp.detach().contiguous())
        H = bse.assemble()
        om, rs, vec = bse.lowest(H, n_eig, n_steps, seed, vectors=True)
        del H
        ctx.bse = bse
        ctx.save_for_backward(vec)
        ctx.mark_non_differentiable(rs)
        return om, rs

    @staticmethod
    def backward(ctx, g_om, g_rs):
        (vec,) = ctx.saved_tensors
        bse = ctx.bse
        Gamma = bse.adjoint_seed(vec, g_om.detach().to(torch.float64).contiguous())
        dW, de = bse.adjoint(Gamma)
        return dW, de, None, None, None, None, None
