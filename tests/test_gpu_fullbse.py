"""Full BSE on the GPU: the coupling block B (bse_assemble_coupling) element by element against
the oracle, the full-BSE spectrum (bse_spectrum_full) against the oracle's paired
eigen-decomposition, the lowest paired excitation energies (bse_lowest_full), the B = 0
limit, and the error raised for an unstable (indefinite) [[A, B], [B*, A*]]."""
import numpy as np
import pytest

import oracle as O
from synth import config_spec, full_bse_spec, make_inputs

from helpers import SPLIT_B, to_dev
from test_gpu_fp64 import RAGGED, REL

pytestmark = pytest.mark.gpu

ETA = 0.1


def _gpu_AB(inp, precision="fp64"):
    from paper_2607_05853_b300.api import BSE
    b = BSE.from_inputs(inp, precision=precision)
    d = to_dev(inp)
    b.interp_W(d["W_R"], d["V0"])
    b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
    A = b.assemble()
    B = b.assemble_coupling()
    b.sync()
    return b, d, A, B


@pytest.mark.parametrize("name", ["cfg0", "ragged", "two_d", "wide", "gamma_only"])
def test_coupling_block_matches_oracle(name):
    inp = make_inputs(config_spec(0) if name == "cfg0" else RAGGED[name])
    ref = O.BSEOracle(inp).coupling()
    b, d, A, B = _gpu_AB(inp)
    B = B.cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(B - ref).max() <= REL * scale
    assert np.abs(B - B.T).max() <= 1e-13 * scale


# split precisions: B has no E_c - E_v diagonal, so its error is bounded relative to max|B|
# itself (tests/helpers.py SPLIT_B, between the measured bf16x3 and bf16x2 errors)


@pytest.mark.parametrize("prec,name", [("bf16x3", "cfg0"), ("bf16x2", "ragged"), ("bf16x3", "wide"),
                                       ("bf16x1", "cfg0"), ("bf16x3", "two_d"), ("tf32x2", "cfg0"),
                                       ("tf32x2", "two_d")])
def test_coupling_block_split_matches_oracle(prec, name):
    inp = make_inputs(config_spec(0) if name == "cfg0" else RAGGED[name])
    ref = O.BSEOracle(inp).coupling()
    b, d, A, B = _gpu_AB(inp, precision=prec)
    B = B.cpu().numpy().astype(np.complex128)
    scale = np.abs(ref).max()
    assert np.abs(B - ref).max() <= SPLIT_B[prec] * scale, (prec, np.abs(B - ref).max() / scale)
    assert np.abs(B - B.T).max() <= SPLIT_B[prec] * scale


def test_full_spectrum_split_odd_dim_matches_oracle():
    """An odd dim (135) takes the single-pass full-read product (k_mmv, complex64) instead of
    the tiled half reads."""
    import dataclasses
    import torch
    spec = dataclasses.replace(RAGGED["ragged"], nv=3, nc=3, dense=(3, 1, 5))
    inp = make_inputs(full_bse_spec(spec))
    orc = O.BSEOracle(inp)
    om = np.linspace(0.0, 12.0, 241)
    ref = O.eps2_full_exact(orc.hamiltonian(), orc.coupling(), orc.dipoles(), om, ETA, orc.prefactor())
    b, d, A, B = _gpu_AB(inp, precision="bf16x3")
    assert b.dim % 2 == 1
    u = b.dipole_vector(d["vel"], d["e_ks"])
    eps = b.spectrum_full(A, B, u, 2 * b.dim, torch.from_numpy(om).cuda(), ETA, orc.prefactor())
    b.sync()
    assert np.linalg.norm(eps.cpu().numpy() - ref) <= 1e-4 * np.linalg.norm(ref)


def test_full_spectrum_split_matches_oracle():
    """bf16x3 A and B (complex64) with the FP64 recursion, full length."""
    import torch
    inp = make_inputs(full_bse_spec(config_spec(0)))
    orc = O.BSEOracle(inp)
    om = np.linspace(0.0, 12.0, 241)
    ref = O.eps2_full_exact(orc.hamiltonian(), orc.coupling(), orc.dipoles(), om, ETA, orc.prefactor())
    b, d, A, B = _gpu_AB(inp, precision="bf16x3")
    u = b.dipole_vector(d["vel"], d["e_ks"])
    eps = b.spectrum_full(A, B, u, 2 * b.dim, torch.from_numpy(om).cuda(), ETA, orc.prefactor())
    b.sync()
    assert np.linalg.norm(eps.cpu().numpy() - ref) <= 1e-4 * np.linalg.norm(ref)


@pytest.mark.parametrize("name", ["cfg0", "ragged", "two_d"])
def test_full_spectrum_full_length_matches_oracle(name):
    """With 2 dim steps the Krylov space is the whole space: the quadrature is exact."""
    import torch
    inp = make_inputs(full_bse_spec(config_spec(0) if name == "cfg0" else RAGGED[name]))
    orc = O.BSEOracle(inp)
    Aref, Bref = orc.hamiltonian(), orc.coupling()
    om = np.linspace(0.0, 12.0, 241)
    ref = O.eps2_full_exact(Aref, Bref, orc.dipoles(), om, ETA, orc.prefactor())
    b, d, A, B = _gpu_AB(inp)
    u = b.dipole_vector(d["vel"], d["e_ks"])
    omega = torch.from_numpy(om).cuda()
    eps = b.spectrum_full(A, B, u, 2 * b.dim, omega, ETA, orc.prefactor())
    b.sync()
    got = eps.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


def test_full_spectrum_krylov_convergence_and_tda_difference():
    """Config-0 full BSE: 300 steps against the exact spectrum (Krylov convergence at eta =
    0.1 eV), and the full spectrum differs from the TDA one by more than that error (B matters)."""
    import torch
    inp = make_inputs(full_bse_spec(config_spec(0)))
    orc = O.BSEOracle(inp)
    Aref, Bref, dref = orc.hamiltonian(), orc.coupling(), orc.dipoles()
    om = np.linspace(0.0, 12.0, 241)
    ref = O.eps2_full_exact(Aref, Bref, dref, om, ETA, orc.prefactor())
    tda = O.eps2_exact(Aref, dref, om, ETA, orc.prefactor())
    b, d, A, B = _gpu_AB(inp)
    u = b.dipole_vector(d["vel"], d["e_ks"])
    eps = b.spectrum_full(A, B, u, 300, torch.from_numpy(om).cuda(), ETA, orc.prefactor())
    b.sync()
    err = np.linalg.norm(eps.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-3
    assert np.linalg.norm(tda - ref) / np.linalg.norm(ref) > 10 * err


def test_full_spectrum_without_coupling_is_tda():
    import torch
    inp = make_inputs(full_bse_spec(RAGGED["ragged"]))
    orc = O.BSEOracle(inp)
    om = np.linspace(0.0, 12.0, 121)
    b, d, A, B = _gpu_AB(inp)
    u = b.dipole_vector(d["vel"], d["e_ks"])
    omega = torch.from_numpy(om).cuda()
    e_full = b.spectrum_full(A, torch.zeros_like(B), u, 2 * b.dim, omega, ETA, orc.prefactor())
    e_tda = b.spectrum(A, u, b.dim, omega, ETA, orc.prefactor())
    b.sync()
    e_full, e_tda = e_full.cpu().numpy(), e_tda.cpu().numpy()
    assert np.abs(e_full - e_tda).max() <= 1e-8 * np.abs(e_tda).max()


def test_lowest_full_matches_oracle():
    inp = make_inputs(full_bse_spec(config_spec(0)))
    orc = O.BSEOracle(inp)
    w, X, Y = O.full_bse_pairs(orc.hamiltonian(), orc.coupling())
    b, d, A, B = _gpu_AB(inp)
    om, rs = b.lowest_full(A, B, 6, 600)
    b.sync()
    om, rs = om.cpu().numpy(), rs.cpu().numpy()
    conv = rs < 1e-6
    assert conv[:3].all()
    assert np.all(np.abs(om[conv] - w[:6][conv]) <= 1e-8 + rs[conv])


def test_indefinite_metric_is_reported():
    """At the calibrated W scale the synthetic config-0 [[A, B], [B*, A*]] has a negative
    eigenvalue (an unstable full BSE): the recursion reports it through bse_sync."""
    import torch
    from paper_2607_05853_b300.api import BseError
    inp = make_inputs(config_spec(0))
    orc = O.BSEOracle(inp)
    b, d, A, B = _gpu_AB(inp)
    u = b.dipole_vector(d["vel"], d["e_ks"])
    b.spectrum_full(A, B, u, 2 * b.dim, torch.linspace(0, 10, 11, dtype=torch.float64, device="cuda"), ETA,
                    orc.prefactor())
    with pytest.raises(BseError, match="not positive definite"):
        b.sync()
    b.sync()  # the error word was cleared: the context stays usable


def test_coupling_rejected_at_finite_Q_and_before_pairs():
    from paper_2607_05853_b300.api import BSE, BseError
    inp = make_inputs(config_spec(0))
    b = BSE.from_inputs(inp, precision="fp64")
    with pytest.raises(BseError):
        b.assemble_coupling()
    b.sync()
