"""Gradients on the 3600-dim monolayer workload (900 k-points, N_aux 240, Nv = Nc = 2) checked
by central finite differences of the GPU's FP64 forward, step 1e-6.

Two scalars, each through its torch.autograd.Function: the sum of the four lowest exciton
energies (Hellmann-Feynman, ExcitonEnergies) and the absorption integral over 1.5-3 eV
(Daleckii-Krein, WindowIntegral).  Perturbed inputs: eight seeded symmetric pairs
W_mu,nu(R), W_nu,mu(-R) (a real W(R) with W(-R) = W(R)^T moves as a pair) and the four
per-band quasiparticle shifts Delta_n (E^QP_n(k) + Delta_n at every k).  The analytic
gradients come from the FP64 forward and from the bf16x3 forward (complex64 H, its Ritz
vectors / Krylov data, FP64 adjoint): the FP64 one must match the differences to the
difference's own accuracy, the split one to 1e-3 of the gradient's scale, the accuracy a
split forward allows (the 1e-6 step lies below split rounding, so the differences run on the
FP64 path)."""
import numpy as np
import pytest

from synth import config_spec, make_inputs

from helpers import to_dev

pytestmark = pytest.mark.gpu

LO, HI, ETA = 1.5, 3.0, 0.1
N_EIG, EIG_STEPS, WIN_STEPS = 4, 400, 1000
STEP = 1e-6


@pytest.fixture(scope="module")
def mono():
    import torch
    from paper_2607_05853_b300.api import BSE
    from paper_2607_05853_b300.grad import ExcitonEnergies, WindowIntegral
    inp = make_inputs(config_spec(4))
    d = to_dev(inp)
    pref = 4.0 * np.pi ** 2 / (3.0 * int(np.prod(inp["dense"])) * float(inp["volume"]))
    grads = {}
    for prec in ("fp64", "bf16x3"):
        b = BSE.from_inputs(inp, precision=prec)
        u = b.dipole_vector(d["vel"], d["e_ks"])
        W = d["W_R"].clone().requires_grad_(True)
        e = d["e_qp"].clone().requires_grad_(True)
        om, _ = ExcitonEnergies.apply(W, e, b, d, N_EIG, EIG_STEPS, 12345)
        om.sum().backward()
        g_eig = (W.grad.cpu().numpy().copy(), e.grad.cpu().numpy().copy())
        W.grad = None
        e.grad = None
        I = WindowIntegral.apply(W, e, b, d, u, WIN_STEPS, LO, HI, ETA, pref)
        I.backward()
        g_win = (W.grad.cpu().numpy().copy(), e.grad.cpu().numpy().copy())
        b.sync()
        grads[prec] = {"eig": g_eig, "win": g_win, "om": om.detach().cpu().numpy(), "I": I.item()}
        if prec == "bf16x3":
            b.close()
        else:
            fp64 = b
            u64 = u
    torch.cuda.synchronize()
    return inp, d, pref, fp64, u64, grads


def _forward(b, d, u, pref, W_R, e_qp):
    """Both scalars from one FP64 assembly of the perturbed inputs."""
    import torch
    b.interp_W(torch.from_numpy(W_R).cuda(), d["V0"])
    b.project_pairs(d["C_R"], d["c_k"], torch.from_numpy(e_qp).cuda())
    H = b.assemble()
    om, _ = b.lowest(H, N_EIG, EIG_STEPS, 12345)
    _, I = b.window_seed(H, u, WIN_STEPS, LO, HI, ETA, pref)
    b.sync()
    return float(om.sum().item()), float(I.item())


def _perturbations(inp):
    """(description, function mapping (W_R, e_qp, s) to perturbed copies, gradient extractor)."""
    RW = inp["R_W"]
    naux = inp["W_R"].shape[1]
    nv = int(inp["nv"])
    rng = np.random.default_rng(20260004)
    out = []
    for _ in range(8):
        r, m, n = int(rng.integers(len(RW))), int(rng.integers(naux)), int(rng.integers(naux))
        rp = [i for i in range(len(RW)) if np.all(RW[i] == -RW[r])][0]
        single = rp == r and m == n

        def pert(W, e, s, r=r, m=m, n=n, rp=rp, single=single):
            W = W.copy()
            W[r, m, n] += s
            if not single:
                W[rp, n, m] += s
            return W, e

        def grad(gW, ge, r=r, m=m, n=n, rp=rp, single=single):
            return gW[r, m, n] + (0.0 if single else gW[rp, n, m])
        out.append((f"W[{r},{m},{n}]", pert, grad))
    for band in range(nv + int(inp["nc"])):
        def pert(W, e, s, band=band):
            e = e.copy()
            e[:, band] += s
            return W, e

        def grad(gW, ge, band=band):
            return ge[:, band].sum()
        out.append((f"Delta_{band}", pert, grad))
    return out


def test_monolayer_gradients_against_central_differences(mono):
    inp, d, pref, b, u, grads = mono
    W0, e0 = np.ascontiguousarray(inp["W_R"]), np.ascontiguousarray(inp["e_qp"])
    rows = []
    for name, pert, grad in _perturbations(inp):
        vals = [_forward(b, d, u, pref, *pert(W0, e0, s)) for s in (STEP, -STEP)]
        fd_eig = (vals[0][0] - vals[1][0]) / (2 * STEP)
        fd_win = (vals[0][1] - vals[1][1]) / (2 * STEP)
        rows.append((name, fd_eig, grad(*grads["fp64"]["eig"]), grad(*grads["bf16x3"]["eig"]),
                     fd_win, grad(*grads["fp64"]["win"]), grad(*grads["bf16x3"]["win"])))
    rows = np.array([r[1:] for r in rows])
    for name, r in zip([p[0] for p in _perturbations(inp)], rows):
        print(name, " ".join(f"{x:+.6e}" for x in r))
    # scales: the largest checked gradient of each scalar
    s_eig, s_win = np.abs(rows[:, 1]).max(), np.abs(rows[:, 4]).max()
    # FP64 analytic vs differences: the difference carries ~1e-13 |value| / 1e-6 of rounding
    assert np.abs(rows[:, 0] - rows[:, 1]).max() <= 1e-5 * s_eig
    assert np.abs(rows[:, 3] - rows[:, 4]).max() <= 1e-4 * s_win
    # split forward (bf16x3) vs the FP64 differences
    assert np.abs(rows[:, 0] - rows[:, 2]).max() <= 1e-3 * s_eig
    assert np.abs(rows[:, 3] - rows[:, 5]).max() <= 1e-3 * s_win
    # shift sum rules of the analytic FP64 gradient: a rigid shift of every conduction band
    # moves each of the four excitons by +1, of every valence band by -1
    nv = int(inp["nv"])
    band_rows = rows[8:]
    assert np.isclose(band_rows[nv:, 1].sum(), N_EIG, atol=1e-8)
    assert np.isclose(band_rows[:nv, 1].sum(), -N_EIG, atol=1e-8)
