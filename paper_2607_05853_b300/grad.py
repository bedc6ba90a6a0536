"""Differentiable lowest exciton energies and windowed absorption integral: torch.autograd
Functions whose forward runs the library's assembly and Lanczos, and whose backward is the
library's hand-written adjoint.

    Omega = ExcitonEnergies.apply(W_R, e_qp, bse, fixed, n_eig, n_steps, seed)
    I = WindowIntegral.apply(W_R, e_qp, bse, fixed, u, n_steps, w_lo, w_hi, eta, prefactor)

W_R ([n_RW][N_aux][N_aux] float64) and e_qp ([N_k][nv+nc] float64) are the differentiable
inputs; `fixed` holds the device tensors V0, C_R, c_k of the same crystal.  The backward
builds the Hellmann-Feynman seed sum_s g_s x_s x_s^dagger from the Ritz vectors of the forward
(bse_adjoint_seed) and contracts it through the assembly (bse_adjoint), recomputing the pair
projections instead of storing them.  WindowIntegral's forward returns
I = int_{w_lo}^{w_hi} eps2(w) dw (Eq. abs_vel, Lorentzian of half width eta) and keeps the
Daleckii-Krein seed Gamma of bse_window_seed (dI = tr(Gamma dH)), which its backward contracts
through bse_adjoint.  u (the start vectors, e.g. from bse_dipole_vector) depends on the
Kohn-Sham energies only, so it is not differentiated.  Only the binding's calls run; the
one multiplication by the incoming scalar gradient is the chain rule.
"""
from __future__ import annotations

import torch

from .api import BSE

__all__ = ["ExcitonEnergies", "WindowIntegral"]


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


class WindowIntegral(torch.autograd.Function):
    @staticmethod
    def forward(ctx, W_R: torch.Tensor, e_qp: torch.Tensor, bse: BSE, fixed: dict, u: torch.Tensor, n_steps: int,
                w_lo: float, w_hi: float, eta: float, prefactor: float):
        bse.interp_W(W_R.detach().contiguous(), fixed["V0"])
        bse.project_pairs(fixed["C_R"], fixed["c_k"], e_qp.detach().contiguous())
        H = bse.assemble()
        Gamma, I = bse.window_seed(H, u, n_steps, w_lo, w_hi, eta, prefactor)
        del H
        ctx.bse = bse
        ctx.save_for_backward(Gamma)
        return I.reshape(())

    @staticmethod
    def backward(ctx, g_I):
        (Gamma,) = ctx.saved_tensors
        dW, de = ctx.bse.adjoint(Gamma)
        g = g_I.detach().to(torch.float64)
        return g * dW, g * de, None, None, None, None, None, None, None, None
