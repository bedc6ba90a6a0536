"""GPU adjoint of the windowed absorption integral (bse_window_seed + bse_adjoint) against
the FP64 oracle: the integral itself, the Daleckii-Krein seed Gamma and the gradients with
respect to W(R) and the quasiparticle energies.  With n_steps = dim the Lanczos subspace is
the whole space, so the Krylov formula is exact and the FP64 path must agree to rounding."""
import numpy as np
import pytest

import oracle as O
from synth import config_spec, make_inputs

from helpers import gpu_hamiltonian
from test_gpu_fp64 import RAGGED

pytestmark = pytest.mark.gpu

LO, HI, ETA = 1.5, 3.0, 0.1


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def cfg0():
    inp = make_inputs(config_spec(0))
    orc = O.BSEOracle(inp)
    H = orc.hamiltonian()
    d = orc.dipoles()
    pref = orc.prefactor()
    G = O.window_seed_exact(H, d, LO, HI, ETA, pref)
    I = O.window_integral(H, d, LO, HI, ETA, pref)
    dW, de = O.grad_from_seed(orc, G)
    return inp, orc, pref, G, I, dW, de


def _gpu_window(inp, precision, n_steps=None, pref=None):
    b, d, H, _ = gpu_hamiltonian(inp, precision=precision)
    u = b.dipole_vector(d["vel"], d["e_ks"])
    G, I = b.window_seed(H, u, n_steps or b.dim, LO, HI, ETA, pref)
    dW, de = b.adjoint(G)
    b.sync()
    return b, G.cpu().numpy(), I.item(), dW.cpu().numpy(), de.cpu().numpy()


def test_window_seed_fp64_full_length_matches_oracle(cfg0):
    inp, orc, pref, G_ref, I_ref, dW_ref, de_ref = cfg0
    b, G, I, dW, de = _gpu_window(inp, "fp64", pref=pref)
    assert abs(I - I_ref) <= 1e-10 * abs(I_ref)
    assert np.linalg.norm(G - G_ref) <= 1e-8 * np.linalg.norm(G_ref)
    assert _rel(dW, dW_ref) <= 1e-8
    assert _rel(de, de_ref) <= 1e-8


def test_window_seed_shift_sum_rule_on_gpu(cfg0):
    """Sum over conduction bands of dI/dE^QP = eps2(lo) - eps2(hi) of the GPU's own spectrum."""
    import torch
    inp, orc, pref, *_ = cfg0
    b, d, H, _ = gpu_hamiltonian(inp, precision="fp64")
    u = b.dipole_vector(d["vel"], d["e_ks"])
    G, I = b.window_seed(H, u, b.dim, LO, HI, ETA, pref)
    dW, de = b.adjoint(G)
    om = torch.tensor([LO, HI], dtype=torch.float64, device="cuda")
    eps = b.spectrum(H, u, b.dim, om, ETA, pref).cpu().numpy()
    b.sync()
    de = de.cpu().numpy()
    assert np.isclose(de[:, orc.nv:].sum(), eps[0] - eps[1], rtol=1e-8)
    assert np.isclose(de[:, :orc.nv].sum(), eps[1] - eps[0], rtol=1e-8)


def test_window_seed_split_forward(cfg0):
    """bf16x3 forward (complex64 H) with the FP64 adjoint: within the split path's accuracy."""
    inp, orc, pref, G_ref, I_ref, dW_ref, de_ref = cfg0
    b, G, I, dW, de = _gpu_window(inp, "bf16x3", pref=pref)
    assert abs(I - I_ref) <= 1e-4 * abs(I_ref)
    assert np.linalg.norm(dW - dW_ref) <= 1e-3 * np.linalg.norm(dW_ref)
    assert np.linalg.norm(de - de_ref) <= 1e-3 * np.linalg.norm(de_ref)


def test_window_integral_autograd_matches_oracle(cfg0):
    """WindowIntegral.apply(...).backward(): the forward's I and the gradients that reach W_R
    and e_qp equal the oracle's exact integral and its Daleckii-Krein gradient (FP64 path,
    Lanczos run to full length), scaled by the incoming gradient."""
    import torch
    from paper_2607_05853_b300.api import BSE
    from paper_2607_05853_b300.grad import WindowIntegral
    from helpers import to_dev
    inp, orc, pref, G_ref, I_ref, dW_ref, de_ref = cfg0
    b = BSE.from_inputs(inp, precision="fp64")
    d = to_dev(inp)
    u = b.dipole_vector(d["vel"], d["e_ks"])
    W = d["W_R"].clone().requires_grad_(True)
    e = d["e_qp"].clone().requires_grad_(True)
    I = WindowIntegral.apply(W, e, b, d, u, b.dim, LO, HI, ETA, pref)
    (2.5 * I).backward()
    assert abs(I.item() - I_ref) <= 1e-10 * abs(I_ref)
    assert _rel(W.grad.cpu().numpy(), 2.5 * dW_ref) <= 1e-8
    assert _rel(e.grad.cpu().numpy(), 2.5 * de_ref) <= 1e-8


@pytest.mark.parametrize("name", ["ragged", "two_d"])
def test_window_seed_ragged_shapes(name):
    inp = make_inputs(RAGGED[name])
    orc = O.BSEOracle(inp)
    H = orc.hamiltonian()
    d, pref = orc.dipoles(), orc.prefactor()
    G_ref = O.window_seed_exact(H, d, LO, HI, ETA, pref)
    I_ref = O.window_integral(H, d, LO, HI, ETA, pref)
    dW_ref, de_ref = O.grad_from_seed(orc, G_ref)
    b, G, I, dW, de = _gpu_window(inp, "fp64", pref=pref)
    assert abs(I - I_ref) <= 1e-9 * max(abs(I_ref), 1e-30)
    assert np.linalg.norm(G - G_ref) <= 1e-7 * np.linalg.norm(G_ref)
    assert _rel(dW, dW_ref) <= 1e-7
    assert _rel(de, de_ref) <= 1e-7


@pytest.mark.slow
def test_window_gradient_monolayer_krylov_convergence():
    """The 3600-dim monolayer workload (FP64 path): the window-integral gradient from 400
    Lanczos steps against the one from 1200 steps (Krylov convergence), with timings."""
    import time
    import torch
    inp = make_inputs(config_spec(4))
    b, d, H, _ = gpu_hamiltonian(inp, precision="fp64")
    u = b.dipole_vector(d["vel"], d["e_ks"])
    pref = O.spectrum_prefactor(b.nk, float(inp["volume"]))
    out = {}
    for m in (400, 1200):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G, I = b.window_seed(H, u, m, LO, HI, ETA, pref)
        dW, de = b.adjoint(G)
        b.sync()
        out[m] = (I.item(), dW.cpu().numpy(), de.cpu().numpy(), time.perf_counter() - t0)
    (I1, w1, e1, t1), (I2, w2, e2, t2) = out[400], out[1200]
    print(f"monolayer window gradient: 400 steps {t1:.2f} s, 1200 steps {t2:.2f} s; I = {I2:.6e}")
    assert abs(I1 - I2) <= 1e-6 * abs(I2)
    assert np.linalg.norm(w1 - w2) <= 1e-4 * np.linalg.norm(w2)
    assert np.linalg.norm(e1 - e2) <= 1e-4 * np.linalg.norm(e2)
