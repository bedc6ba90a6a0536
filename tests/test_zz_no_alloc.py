"""bse_spectrum_static: the allocation-free spectrum, for callers that cannot allocate
device memory (a host application that owns the device pool, or a GPU already at its
memory limit).  It must give what bse_spectrum gives, call after call, while its scratch
lives in one fixed device array that every call reuses.

This file is collected last on purpose, so that a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle as O
from synth import config_spec, make_inputs

from helpers import gpu_hamiltonian

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_static_spectrum_matches_allocating_spectrum_twice(prec):
    import torch
    from paper_2607_05853_b300.api import BseError
    inp = make_inputs(config_spec(0))
    orc = O.BSEOracle(inp)
    b, d, H, _ = gpu_hamiltonian(inp, precision=prec)
    u = b.dipole_vector(d["vel"], d["e_ks"])
    om = torch.linspace(0.0, 10.0, 301, dtype=torch.float64, device="cuda")
    n = 200
    ref_ab = torch.empty((3, 3, n), dtype=torch.float64, device="cuda")
    ref = b.spectrum(H, u, n, om, 0.1, orc.prefactor(), ab=ref_ab)
    b.sync()
    ref, ref_ab = ref.cpu().numpy(), ref_ab.cpu().numpy()
    for call in range(2):  # the second call finds the previous call's contents in the array
        eps = torch.full_like(om, float("nan"))
        ab = torch.full((3, 3, n), float("nan"), dtype=torch.float64, device="cuda")
        b.spectrum_static(H, u, n, om, 0.1, orc.prefactor(), eps, ab)
        b.sync()
        eps, ab = eps.cpu().numpy(), ab.cpu().numpy()
        assert np.all(np.isfinite(eps)), call
        assert np.abs(eps - ref).max() <= 1e-9 * np.abs(ref).max(), call
        assert np.allclose(ab, ref_ab, rtol=0, atol=1e-10 * np.abs(ref_ab).max()), call
    if prec == "bf16x3":
        # full length with three polarisations needs ~75 MB of scratch here: refused up front
        eps = torch.empty_like(om)
        with pytest.raises(BseError, match="EINVAL"):
            b.spectrum_static(H, u, b.dim, om, 0.1, orc.prefactor(), eps)
    b.close()
