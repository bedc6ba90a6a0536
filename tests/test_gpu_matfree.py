"""Matrix-free Haydock spectrum (bse_spectrum_matfree: every Lanczos product recomputed from
the pair tables, H never stored) against the stored-H spectrum of the same context and
against the oracle."""
import numpy as np
import pytest

import oracle as O
from synth import config_spec, make_inputs

from helpers import to_dev
from synth import CrystalSpec
from synth.crystal import _fcc
from test_gpu_fp64 import RAGGED

pytestmark = pytest.mark.gpu

ETA = 0.1

# Nv = 2 with N_aux <= 160: the fused kernel's matrix-free form with two-lane j sums (cfg0 has
# Nv = 4; ragged, two_d and wide take the unfused block application)
NV2 = CrystalSpec("nv2", _fcc(5.43), np.array([[0, 0, 0], [0.25, 0.25, 0.25]]), (7, 7), (11, 13), (2, 1, 1),
                  (3, 2, 2), 2, 6, 2718, r_max=1.0)


def _ctx(inp, precision="bf16x3", Q=None):
    import torch
    from paper_2607_05853_b300.api import BSE
    b = BSE.from_inputs(inp, precision=precision)
    d = to_dev(inp)
    if Q is not None:
        b.set_momentum(Q, torch.from_numpy(np.ascontiguousarray(inp["V_R"], np.float64)).cuda())
        b.interp_W(d["W_R"], None)
    else:
        b.interp_W(d["W_R"], d["V0"])
    b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
    return b, d


@pytest.mark.parametrize("name", ["cfg0", "nv2", "ragged", "wide", "two_d"])
def test_matfree_lanczos_matches_stored_H(name):
    """Same recursion coefficients (a_j, b_j) as the stored complex64 H: the two differ only in
    where the FP32-accurate elements are rounded."""
    import torch
    inp = make_inputs(config_spec(0) if name == "cfg0" else NV2 if name == "nv2" else RAGGED[name])
    b, d = _ctx(inp)
    H = b.assemble()
    u = b.dipole_vector(d["vel"], d["e_ks"])
    n = min(60, b.dim)
    om = torch.linspace(0.0, 10.0, 201, dtype=torch.float64, device="cuda")
    ab1 = torch.zeros((3, 3, n), dtype=torch.float64, device="cuda")
    ab2 = torch.zeros_like(ab1)
    e1 = b.spectrum(H, u, n, om, ETA, 1.0, ab=ab1)
    e2 = b.spectrum_matfree(u, n, om, ETA, 1.0, ab=ab2)
    b.sync()
    a1, a2 = ab1.cpu().numpy(), ab2.cpu().numpy()
    scale = np.abs(a1[:, :2]).max()
    assert np.abs(a1[:, :2, :20] - a2[:, :2, :20]).max() <= 1e-5 * scale
    assert np.linalg.norm((e1 - e2).cpu().numpy()) <= 1e-5 * np.linalg.norm(e1.cpu().numpy())


def test_matfree_full_length_matches_oracle():
    import torch
    inp = make_inputs(config_spec(0))
    orc = O.BSEOracle(inp)
    om_np = np.linspace(0.0, 10.0, 201)
    ref = O.eps2_exact(orc.hamiltonian(), orc.dipoles(), om_np, ETA, orc.prefactor())
    b, d = _ctx(inp)
    u = b.dipole_vector(d["vel"], d["e_ks"])
    eps = b.spectrum_matfree(u, b.dim, torch.from_numpy(om_np).cuda(), ETA, orc.prefactor())
    b.sync()
    assert np.linalg.norm(eps.cpu().numpy() - ref) <= 1e-4 * np.linalg.norm(ref)


def test_matfree_finite_momentum_matches_stored_H():
    """At Q != 0 (relabelled tables, complex exchange V) the products are those of H(Q)."""
    import torch
    inp = make_inputs(config_spec(0))
    b, d = _ctx(inp, Q=(1, 2, 0))
    H = b.assemble()
    g = torch.Generator(device="cpu").manual_seed(3)
    u = torch.complex(torch.randn(b.dim, generator=g, dtype=torch.float64),
                      torch.randn(b.dim, generator=g, dtype=torch.float64)).cuda().reshape(1, -1)
    om = torch.linspace(0.0, 12.0, 121, dtype=torch.float64, device="cuda")
    e1 = b.spectrum(H, u, 80, om, ETA, 1.0)
    e2 = b.spectrum_matfree(u, 80, om, ETA, 1.0)
    b.sync()
    assert np.linalg.norm((e1 - e2).cpu().numpy()) <= 1e-5 * np.linalg.norm(e1.cpu().numpy())


def test_matfree_rejects_fp64_and_order():
    import torch
    from paper_2607_05853_b300.api import BSE, BseError
    inp = make_inputs(config_spec(0))
    b = BSE.from_inputs(inp, precision="bf16x3")
    u = torch.zeros((1, b.dim), dtype=torch.complex128, device="cuda")
    om = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(BseError):            # before project_pairs
        b.spectrum_matfree(u, 10, om, ETA, 1.0)
    f = BSE.from_inputs(inp, precision="fp64")
    d = to_dev(inp)
    f.interp_W(d["W_R"], d["V0"])
    f.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
    with pytest.raises(BseError):            # FP64 context
        f.spectrum_matfree(u, 10, om, ETA, 1.0)
    f.sync()
