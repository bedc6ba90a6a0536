"""k-offset averaging of the absorption spectrum (§IV, convergence with k-point sampling).

Independent calculations on dense meshes shifted away from Gamma are averaged with the
weights of the symmetry-reduced classes of a 3x3x3 grid of offsets (in units of the dense
mesh spacing): four offsets with weights 1/27, 8/27, 6/27 and 12/27.  Each offset is its own
system (its own band coefficients and energies at the shifted k-points); W(q) does not
depend on the offset because q = k1 - k2 does not.  The assemblies of all offsets run as one
CUDA graph (bse_batch_assemble) and the spectra are accumulated on the device with their
weights (bse_spectrum_add).
"""
from __future__ import annotations

import torch

from .api import batch_assemble

OFFSETS = ((0.0, 0.0, 0.0), (1.0 / 3, 0.0, 0.0), (1.0 / 3, 1.0 / 3, 0.0), (2.0 / 3, 1.0 / 3, 0.0))
WEIGHTS = (1.0 / 27, 8.0 / 27, 6.0 / 27, 12.0 / 27)


def offset_average(systems, Hs, dipoles, omega: torch.Tensor, n_steps: int, eta: float, prefactors,
                   weights=WEIGHTS, batched: bool = True) -> torch.Tensor:
    """sum_o weights[o] * eps2_o(omega) for the systems of the shifted meshes.

    systems: BSE contexts, one per offset, each past project_pairs (set up with that offset's
    k_offset); Hs: their H buffers; dipoles: their start vectors u (from dipole_vector);
    prefactors: their spectrum prefactors.  batched=False assembles the systems one by one."""
    if not (len(systems) == len(Hs) == len(dipoles) == len(prefactors) == len(weights)):
        raise ValueError("offset_average: one system, H, dipole vector, prefactor and weight per offset")
    if batched:
        split = all(b.precision != "fp64" and b.precision == systems[0].precision for b in systems)
        batch_assemble(systems, Hs, schedule="worklist" if split else "chains")
    else:
        for b, H in zip(systems, Hs):
            b.assemble(H)
    acc = torch.zeros(omega.numel(), dtype=torch.float64, device=omega.device)
    for b, H, u, pref, w in zip(systems, Hs, dipoles, prefactors, weights):
        b.spectrum_add(H, u, min(n_steps, b.dim), omega, eta, pref, w, acc)
    return acc
