"""bse_spectrum_static: the allocation-free spectrum, for callers that cannot allocate
device memory (a host application that owns the device pool, or a GPU already at its
memory limit).  It must give what bse_spectrum gives, call after call, while its scratch
lives in one fixed device array that every call reuses and no call allocates.

Consecutive calls differ (a larger call, then a smaller one on a different H with other
n_pol / n_steps), so a value left in the shared array by the previous call cannot pass for a
fresh one.  The odd-dim split case takes the full-read product instead of the half-read one.

This file is collected last on purpose, so that a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from synth import config_spec, make_inputs

from helpers import gpu_hamiltonian

pytestmark = pytest.mark.gpu


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _outputs(u, n_steps, om):
    import torch
    return (torch.empty_like(om), torch.empty((u.shape[0], 3, n_steps), dtype=torch.float64, device="cuda"))


def _check(b, H, u, n_steps, om, pref, ref_eps, ref_ab, out):
    eps, ab = out
    eps.fill_(float("nan"))
    ab.fill_(float("nan"))
    b.spectrum_static(H, u, n_steps, om, 0.1, pref, eps, ab)
    b.sync()
    eps, ab = eps.cpu().numpy(), ab.cpu().numpy()
    assert np.all(np.isfinite(eps))
    assert np.abs(eps - ref_eps).max() <= 1e-9 * np.abs(ref_eps).max()
    assert np.allclose(ab, ref_ab, rtol=0, atol=1e-10 * np.abs(ref_ab).max())


def _reference(b, H, u, n_steps, om, pref):
    import torch
    ab = torch.empty((u.shape[0], 3, n_steps), dtype=torch.float64, device="cuda")
    eps = b.spectrum(H, u, n_steps, om, 0.1, pref, ab=ab)
    b.sync()
    return eps.cpu().numpy(), ab.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_static_spectrum_matches_allocating_spectrum_twice(prec):
    import torch
    from paper_2607_05853_b300.api import BseError
    om = torch.linspace(0.0, 10.0, 301, dtype=torch.float64, device="cuda")
    # two systems: the tiny workload and the same crystal with another seed and a 3x4x4 mesh
    inp1 = make_inputs(config_spec(0))
    inp2 = make_inputs(dataclasses.replace(config_spec(0), seed=4711, dense=(3, 4, 4)))
    b1, d1, H1, _ = gpu_hamiltonian(inp1, precision=prec)
    b2, d2, H2, _ = gpu_hamiltonian(inp2, precision=prec)
    u1 = b1.dipole_vector(d1["vel"], d1["e_ks"])
    u2 = b2.dipole_vector(d2["vel"], d2["e_ks"])[1:2].contiguous()   # one polarisation
    p1, p2 = O.BSEOracle(inp1).prefactor(), O.BSEOracle(inp2).prefactor()
    ref1 = _reference(b1, H1, u1, 200, om, p1)
    ref2 = _reference(b2, H2, u2, 57, om, p2)
    out1, out2 = _outputs(u1, 200, om), _outputs(u2, 57, om)
    # first call: looks up the array's address (and loads the kernels it needs)
    _check(b1, H1, u1, 200, om, p1, *ref1, out1)
    free0 = _free_bytes()
    _check(b2, H2, u2, 57, om, p2, *ref2, out2)      # smaller call on another H after a larger one
    _check(b1, H1, u1, 200, om, p1, *ref1, out1)     # and the larger one again
    assert _free_bytes() == free0                    # no call allocated device memory
    if prec == "bf16x3":
        # full length with three polarisations needs ~75 MB of scratch here: refused up front
        eps = torch.empty_like(om)
        with pytest.raises(BseError, match="EINVAL"):
            b1.spectrum_static(H1, u1, b1.dim, om, 0.1, p1, eps)
    b1.close()
    b2.close()


def test_static_spectrum_odd_dim_split():
    """An odd dim (135) on the split path: complex64 H through the full-read product."""
    import torch
    from test_gpu_fp64 import RAGGED
    inp = make_inputs(dataclasses.replace(RAGGED["ragged"], nv=3, nc=3, dense=(3, 1, 5)))
    b, d, H, _ = gpu_hamiltonian(inp, precision="bf16x3")
    assert b.dim % 2 == 1
    u = b.dipole_vector(d["vel"], d["e_ks"])
    om = torch.linspace(0.0, 12.0, 241, dtype=torch.float64, device="cuda")
    pref = O.BSEOracle(inp).prefactor()
    ref = _reference(b, H, u, 100, om, pref)
    out = _outputs(u, 100, om)
    for _ in range(2):
        _check(b, H, u, 100, om, pref, *ref, out)
    b.close()
