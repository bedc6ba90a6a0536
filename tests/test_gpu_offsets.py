"""k-offset averaging on the GPU (four shifted dense meshes assembled as one CUDA graph,
spectra accumulated with the paper's weights through bse_spectrum_add) against the oracle's
weighted sum of exact spectra."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from synth import config_spec, make_inputs

from helpers import to_dev

pytestmark = pytest.mark.gpu

ETA = 0.1


def _systems(precision):
    from paper_2607_05853_b300.api import BSE
    from paper_2607_05853_b300 import offsets
    base = config_spec(0)
    inps = [make_inputs(dataclasses.replace(base, k_offset=o)) for o in offsets.OFFSETS]
    systems, us, prefs = [], [], []
    for inp in inps:
        b = BSE.from_inputs(inp, precision=precision)
        d = to_dev(inp)
        b.interp_W(d["W_R"], d["V0"])
        b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
        us.append(b.dipole_vector(d["vel"], d["e_ks"]))
        prefs.append(O.spectrum_prefactor(b.nk, float(inp["volume"])))
        systems.append(b)
    return inps, systems, us, prefs


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("bf16x3", 1e-4)])
def test_offset_average_matches_oracle(precision, tol):
    import torch
    from paper_2607_05853_b300 import offsets
    from paper_2607_05853_b300.api import batch_release
    inps, systems, us, prefs = _systems(precision)
    Hs = [torch.empty((b.dim, b.dim), dtype=b.h_dtype, device="cuda") for b in systems]
    om = torch.linspace(0.0, 10.0, 401, dtype=torch.float64, device="cuda")
    avg = offsets.offset_average(systems, Hs, us, om, systems[0].dim, ETA, prefs)
    torch.cuda.synchronize()
    got = avg.cpu().numpy()
    batch_release()
    for b in systems:
        b.sync()
    ref = O.offset_average_eps2(inps, offsets.WEIGHTS, om.cpu().numpy(), ETA)
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


def test_offset_average_unbatched_equals_batched():
    """The graph-batched assembly and the one-by-one assembly give the same average."""
    import torch
    from paper_2607_05853_b300 import offsets
    from paper_2607_05853_b300.api import batch_release
    inps, systems, us, prefs = _systems("bf16x3")
    om = torch.linspace(0.0, 10.0, 201, dtype=torch.float64, device="cuda")
    H1 = [torch.empty((b.dim, b.dim), dtype=b.h_dtype, device="cuda") for b in systems]
    H2 = [torch.empty((b.dim, b.dim), dtype=b.h_dtype, device="cuda") for b in systems]
    a1 = offsets.offset_average(systems, H1, us, om, 300, ETA, prefs, batched=True)
    a2 = offsets.offset_average(systems, H2, us, om, 300, ETA, prefs, batched=False)
    torch.cuda.synchronize()
    batch_release()
    assert torch.equal(a1, a2)
