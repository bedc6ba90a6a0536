"""The paper's largest dense mesh (21 x 21 x 21 k-points, the meshes of the Si and MgO spectra
of §IV, with 4 + 4 bands) on the 27648-dim workload's cell: dim 148176, H 176 GB complex64
held in HBM, assembled in the precision the benchmark times (bf16x3).  Sampled blocks
against the oracle (every index of the path past 2^31 elements of H), the largest k-point
indices included, with the full-size split bounds; then a short three-polarisation Haydock
recursion on the stored H (finite, non-negative spectrum, no early stop)."""
import dataclasses
import gc

import numpy as np
import pytest

import oracle as O
from synth import config_spec, make_inputs

from helpers import SPLIT_OFF_FULL, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.slow
def test_paper_scale_mesh21_sampled_blocks_and_spectrum():
    import torch
    from paper_2607_05853_b300.api import BSE
    gc.collect()
    torch.cuda.empty_cache()
    inp = make_inputs(dataclasses.replace(config_spec(2), dense=(21, 21, 21), name="mesh21"))
    orc = O.BSEOracle(inp)
    nk, n = orc.nk, orc.nvc
    b = BSE.from_inputs(inp, precision="bf16x3")
    assert b.dim == 148176
    d = to_dev(inp)
    b.interp_W(d["W_R"], d["V0"])
    b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
    H = torch.empty((b.dim, b.dim), dtype=torch.complex64, device="cuda")
    b.assemble(H)
    b.sync()
    rng = np.random.default_rng(148176)
    pairs = [(0, 0), (nk - 1, nk - 1), (nk - 1, 0), (0, nk - 1), (4630, 4631)]
    pairs += [tuple(int(x) for x in rng.integers(0, nk, 2)) for _ in range(8)]
    off = so = dg = sd = 0.0
    for k1, k2 in pairs:
        ref = orc.block(k1, k2)
        got = H[k1 * n:(k1 + 1) * n, k2 * n:(k2 + 1) * n].cpu().numpy().astype(np.complex128)
        eye = np.eye(n, dtype=bool) if k1 == k2 else np.zeros((n, n), bool)
        err = np.abs(got - ref)
        off, so = max(off, err[~eye].max()), max(so, np.abs(ref[~eye]).max())
        if k1 == k2:
            dg, sd = max(dg, err[eye].max()), max(sd, np.abs(ref[eye]).max())
    assert off / so <= SPLIT_OFF_FULL["bf16x3"], off / so
    assert dg / sd <= 1.2e-7, dg / sd
    u = b.dipole_vector(d["vel"], d["e_ks"])
    om = torch.linspace(0.0, 10.0, 201, dtype=torch.float64, device="cuda")
    ab = torch.zeros((3, 3, 40), dtype=torch.float64, device="cuda")
    eps = b.spectrum(H, u, 40, om, 0.1, orc.prefactor(), ab=ab)
    b.sync()
    eps, ab = eps.cpu().numpy(), ab.cpu().numpy()
    assert np.all(np.isfinite(eps)) and eps.min() >= 0.0 and eps.max() > 0.0
    assert np.all(ab[:, 1, :39] > 0.0)   # every beta_j of the 40 steps positive: no early stop
    del H
    b.close()
    torch.cuda.empty_cache()
