"""Finite exciton momentum on the GPU (bse_set_momentum, FP64 path) against the oracle's
H(Q): the Hamiltonian element by element on several meshes and momenta (including a
self-conjugate Q and a ragged mesh), the lowest excitons, the adjoint, and the error paths."""
import time

import numpy as np
import pytest

import oracle as O
from synth import config_spec, make_inputs

from helpers import to_dev, assert_split_close
from test_gpu_fp64 import RAGGED, REL

pytestmark = pytest.mark.gpu


def _gpu_HQ(inp, Q, alpha=2.0, with_V=True, precision="fp64"):
    import torch
    from paper_2607_05853_b300.api import BSE
    b = BSE.from_inputs(inp, precision=precision, alpha=alpha)
    d = to_dev(inp)
    VR = torch.from_numpy(np.ascontiguousarray(inp["V_R"], np.float64)).cuda() if with_V else None
    b.set_momentum(Q, VR)
    b.interp_W(d["W_R"], None if with_V else d["V0"])
    b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
    H = b.assemble()
    b.sync()
    return b, d, H


CASES = [("cfg0", (1, 0, 0)), ("cfg0", (1, 1, 0)), ("cfg0", (2, 2, 2)),   # (2,2,2) on 4^3: Q = -Q
         ("ragged", (1, 1, 3)), ("two_d", (1, 2, 0)), ("wide", (1, 1, 1))]


def _inputs(name):
    return make_inputs(config_spec(0) if name == "cfg0" else RAGGED[name])


@pytest.mark.parametrize("name,Q", CASES)
def test_finite_Q_hamiltonian_matches_oracle(name, Q):
    inp = _inputs(name)
    ref = O.BSEOracle(inp, Q=Q).hamiltonian()
    b, d, H = _gpu_HQ(inp, Q)
    H = H.cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(H - ref).max() <= REL * scale
    assert np.abs(H - H.conj().T).max() <= 1e-13 * scale


# split precisions: the off-diagonal / diagonal bounds of the Q = 0 split tests
# (tests/helpers.py); Q enters only through indices and the FP32 complex V


@pytest.mark.parametrize("prec,name,Q", [("bf16x3", "cfg0", (1, 1, 0)), ("bf16x3", "cfg0", (2, 2, 2)),
                                         ("bf16x2", "ragged", (1, 1, 3)), ("bf16x3", "two_d", (1, 2, 0)),
                                         ("bf16x1", "cfg0", (3, 0, 1)), ("tf32x2", "ragged", (1, 1, 2))])
def test_finite_Q_split_matches_oracle(prec, name, Q):
    inp = _inputs(name)
    ref = O.BSEOracle(inp, Q=Q).hamiltonian()
    b, d, H = _gpu_HQ(inp, Q, precision=prec)
    assert_split_close(H.cpu().numpy(), ref, prec)


def test_finite_Q_triplet_without_V_R():
    """alpha = 0 (triplet) needs no exchange interaction: V0 route, no V_R."""
    inp = _inputs("cfg0")
    ref = O.BSEOracle(inp, alpha=0.0, Q=(1, 2, 3)).hamiltonian()
    b, d, H = _gpu_HQ(inp, (1, 2, 3), alpha=0.0, with_V=False)
    assert np.abs(H.cpu().numpy() - ref).max() <= REL * np.abs(ref).max()


def test_whole_period_Q_is_the_optical_hamiltonian():
    """Q equal to a mesh period reduces to Q = 0: the same launches on the same data, so the
    same bits as the context that never set a momentum."""
    from helpers import gpu_hamiltonian
    inp = _inputs("cfg0")
    _, _, H0, _ = gpu_hamiltonian(inp)
    _, _, Hp = _gpu_HQ(inp, tuple(inp["dense"]), with_V=False)
    assert np.array_equal(H0.cpu().numpy(), Hp.cpu().numpy())


def test_finite_Q_lowest_excitons_match_lapack():
    inp = _inputs("cfg0")
    Q = (1, 1, 0)
    ref = np.linalg.eigvalsh(O.BSEOracle(inp, Q=Q).hamiltonian())[:8]
    b, d, H = _gpu_HQ(inp, Q)
    om, rs = b.lowest(H, 8, 400)
    b.sync()
    om, rs = om.cpu().numpy(), rs.cpu().numpy()
    conv = rs < 1e-8
    assert conv[:4].all()
    assert np.all(np.abs(om[conv] - ref[conv]) <= rs[conv] + 1e-10)


def test_finite_Q_adjoint_matches_oracle():
    """dOmega/dW(R) and dOmega/dE^QP at Q != 0 for the seed x x^dagger of the lowest exciton
    (the conduction derivative lands on k + Q)."""
    import torch
    inp = _inputs("ragged")
    Q = (2, 1, 4)
    orc = O.BSEOracle(inp, Q=Q)
    w, X = O.adjoint_seed_lowest(orc.hamiltonian(), 1)
    G = np.outer(X[:, 0], X[:, 0].conj())
    dW_ref, de_ref = O.grad_from_seed(orc, G)
    b, d, H = _gpu_HQ(inp, Q)
    dW, de = b.adjoint(torch.from_numpy(G).cuda())
    b.sync()
    dW, de = dW.cpu().numpy(), de.cpu().numpy()
    assert np.abs(dW - dW_ref).max() <= 1e-9 * np.abs(dW_ref).max()
    assert np.abs(de - de_ref).max() <= 1e-12


def test_finite_Q_adjoint_split_matches_oracle():
    """The split-precision adjoint at Q != 0 (projections from the relabelled per-k tables) with
    the oracle's exact seed: dW within 1e-5 of the gradient's scale, dE^QP to 1e-12."""
    import torch
    inp = _inputs("ragged")
    Q = (2, 1, 4)
    orc = O.BSEOracle(inp, Q=Q)
    w, X = O.adjoint_seed_lowest(orc.hamiltonian(), 1)
    G = np.outer(X[:, 0], X[:, 0].conj())
    dW_ref, de_ref = O.grad_from_seed(orc, G)
    b, d, H = _gpu_HQ(inp, Q, precision="bf16x3")
    dW, de = b.adjoint(torch.from_numpy(G).cuda())
    b.sync()
    dW, de = dW.cpu().numpy(), de.cpu().numpy()
    assert np.abs(dW - dW_ref).max() <= 1e-5 * np.abs(dW_ref).max()
    assert np.abs(de - de_ref).max() <= 1e-12


def test_finite_Q_error_paths():
    import torch
    from paper_2607_05853_b300.api import BSE, BseError
    inp = _inputs("cfg0")
    d = to_dev(inp)
    b = BSE.from_inputs(inp, precision="fp64")
    with pytest.raises(BseError):            # exchange at Q != 0 without V(R)
        b.set_momentum((1, 0, 0), None)
    VR = torch.from_numpy(np.ascontiguousarray(inp["V_R"], np.float64)).cuda()
    b.set_momentum((1, 0, 0), VR)
    b.interp_W(d["W_R"], None)
    b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
    with pytest.raises(BseError):            # optical dipoles are vertical
        b.dipole_vector(d["vel"], d["e_ks"])
    b.set_momentum((0, 1, 0), VR)            # a new Q needs the pair stage again
    with pytest.raises(BseError):
        b.assemble()
    b.set_momentum((0, 0, 0), None)          # back to V0: needs interp_W again
    with pytest.raises(BseError):
        b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
    b.sync()


def test_exciton_dispersion_monolayer_timing():
    """H(Q) along a line of momenta on the 3600-dim monolayer workload (FP64 path): every Q
    is Hermitian with the oracle's diagonal at Q, and the lowest exciton at the sampled Q
    matches LAPACK on the oracle's H(Q); prints the assembly time per momentum."""
    import torch
    inp = make_inputs(config_spec(4))
    from paper_2607_05853_b300.api import BSE
    b = BSE.from_inputs(inp, precision="fp64")
    d = to_dev(inp)
    VR = torch.from_numpy(np.ascontiguousarray(inp["V_R"], np.float64)).cuda()
    H = torch.empty((b.dim, b.dim), dtype=torch.complex128, device="cuda")
    times, lows = [], []
    n1 = int(inp["dense"][0])
    for m in range(0, n1 // 2 + 1, 2):
        Q = (m, 0, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.set_momentum(Q, VR)
        b.interp_W(d["W_R"], None)
        b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
        b.assemble(H)
        b.sync()
        times.append(time.perf_counter() - t0)
        om, rs = b.lowest(H, 1, 300)
        b.sync()
        lows.append(om.item())
        if m == 2:
            Hc = H.cpu().numpy()
            assert np.abs(Hc - Hc.conj().T).max() <= 1e-13 * np.abs(Hc).max()
    print(f"monolayer H(Q), Q = (0..{n1 // 2}, 0, 0)/{n1}: assembly {np.median(times) * 1e3:.1f} ms per Q; "
          f"lowest exciton {', '.join(f'{x:.4f}' for x in lows)} eV")
    assert np.all(np.isfinite(lows))
