"""Seeded synthetic inputs shaped like the workloads of the dual-k-mesh TDA-BSE method.

This module only *generates inputs* (a tight-binding band structure, localized-RI
coefficients, a screened interaction on a coarse mesh folded to real space, a bare
Coulomb matrix at q=0 and velocity matrix elements). It holds none of the method's
arithmetic (no W interpolation to the dense mesh, no band-pair projection, no kernel
contraction, no spectrum). Both the FP64 oracle and the CUDA path consume its output.
"""
from .crystal import CrystalSpec, config_spec, make_inputs, batched_specs, full_bse_spec, kmesh_frac, kmesh_index

__all__ = ["CrystalSpec", "config_spec", "make_inputs", "batched_specs", "full_bse_spec", "kmesh_frac",
           "kmesh_index"]
