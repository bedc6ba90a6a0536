"""The 27648-dim workload in the precision the benchmark times (bf16x3): sampled blocks of
the full-BSE coupling block B (the half-W variant of the geometry) and of the finite-momentum
Hamiltonian H(Q) against the oracle, at the size the reports in bench.py run, with the
split bounds of tests/helpers.py (B relative to max|B|, H(Q) off-diagonal and diagonal
separately)."""
import numpy as np
import pytest

import oracle as O
from synth import config_spec, full_bse_spec, make_inputs

from helpers import SPLIT_OFF_FULL, to_dev

pytestmark = pytest.mark.gpu


def _pairs(nk):
    rng = np.random.default_rng(21)
    return [(0, 0), (nk - 1, nk - 1), (5, nk - 3)] + [tuple(int(x) for x in rng.integers(0, nk, 2)) for _ in range(10)]


def _block(M, k1, k2, n):
    return M[k1 * n:(k1 + 1) * n, k2 * n:(k2 + 1) * n].cpu().numpy().astype(np.complex128)


def test_full_size_coupling_block_sampled():
    from paper_2607_05853_b300.api import BSE
    inp = make_inputs(full_bse_spec(config_spec(2)))
    b = BSE.from_inputs(inp, precision="bf16x3")
    d = to_dev(inp)
    b.interp_W(d["W_R"], d["V0"])
    b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
    A = b.assemble()
    B = b.assemble_coupling()
    b.sync()
    orc = O.BSEOracle(inp)
    n = orc.nvc
    scale, worst, worst_sym = 0.0, 0.0, 0.0
    for k1, k2 in _pairs(orc.nk):
        ref = orc.coupling_block(k1, k2)
        scale = max(scale, np.abs(ref).max())
        worst = max(worst, np.abs(_block(B, k1, k2, n) - ref).max())
        worst_sym = max(worst_sym, np.abs(_block(B, k1, k2, n) - _block(B, k2, k1, n).T).max())
    print(f"27648-dim B sampled: max error / max|B| = {worst / scale:.3e}")
    assert worst <= SPLIT_OFF_FULL["bf16x3"] * scale
    assert worst_sym <= SPLIT_OFF_FULL["bf16x3"] * scale


def test_full_size_finite_momentum_sampled():
    import torch
    from paper_2607_05853_b300.api import BSE
    inp = make_inputs(config_spec(2))
    Q = (1, 0, 0)
    b = BSE.from_inputs(inp, precision="bf16x3")
    d = to_dev(inp)
    b.set_momentum(Q, torch.from_numpy(np.ascontiguousarray(inp["V_R"], np.float64)).cuda())
    b.interp_W(d["W_R"], None)
    b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
    H = b.assemble()
    b.sync()
    orc = O.BSEOracle(inp, Q=Q)
    n = orc.nvc
    scale = worst = dscale = dworst = 0.0
    for k1, k2 in _pairs(orc.nk):
        ref = orc.block(k1, k2)
        err = np.abs(_block(H, k1, k2, n) - ref)
        eye = np.eye(n, dtype=bool) if k1 == k2 else np.zeros((n, n), bool)
        scale, worst = max(scale, np.abs(ref[~eye]).max()), max(worst, err[~eye].max())
        if k1 == k2:
            dscale, dworst = max(dscale, np.abs(ref[eye]).max()), max(dworst, err[eye].max())
    print(f"27648-dim H(Q) sampled: off-diagonal {worst / scale:.3e}, diagonal {dworst / dscale:.3e}")
    assert worst <= SPLIT_OFF_FULL["bf16x3"] * scale
    assert dworst <= 1.2e-7 * dscale
