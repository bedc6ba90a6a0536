"""Batching of uneven crystals as one CUDA graph (bse_batch_assemble, both schedules: the work
list of grouped tensor-core launches and the two concurrent chains) and the tile autotuner
(bse_autotune): each system's H must equal its unbatched assembly exactly (same kernels, same
tiles, same order of the updates of each element), match the oracle within the split
tolerance, and stay the same on graph replay."""
import numpy as np
import pytest

import oracle as O
from synth import CrystalSpec, batched_specs, make_inputs
from synth.crystal import _fcc, _hex

from helpers import assert_split_close, to_dev

pytestmark = pytest.mark.gpu

# Sanity bound of the sampled blocks of the 16 crystals relative to their largest off-diagonal
# element (measured up to 3.6e-6); the discriminating split bounds are tests/test_gpu_split.py's.
SAMPLED_OFF = 1e-5

SMALL = [
    CrystalSpec("u0", _fcc(5.43), np.array([[0, 0, 0], [0.25, 0.25, 0.25]]), (4, 4), (20, 20), (2, 2, 2), (4, 4, 4),
                4, 4, 11),
    CrystalSpec("u1", np.eye(3) * 4.2, np.zeros((1, 3)), (9,), (37,), (2, 2, 1), (3, 3, 2), 2, 2, 12, r_max=1.5),
    CrystalSpec("u2", _hex(3.3, 6.0), np.array([[0, 0, 0], [1 / 3, 2 / 3, 0.5], [2 / 3, 1 / 3, 0.25]]), (4, 3, 5),
                (11, 9, 14), (2, 1, 1), (4, 2, 1), 2, 4, 13, r_max=1.0),
    CrystalSpec("u3", np.eye(3) * 5.0, np.array([[0, 0, 0], [0.5, 0.5, 0.5]]), (6, 7), (30, 25), (1, 1, 1),
                (2, 2, 3), 6, 6, 14, r_max=1.0),
]


def _setup(specs, prec="bf16x3"):
    import torch
    from paper_2607_05853_b300.api import BSE
    systems = []
    for sp in specs:
        inp = make_inputs(sp)
        b = BSE.from_inputs(inp, precision=prec)
        d = to_dev(inp)
        b.interp_W(d["W_R"], d["V0"])
        b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
        systems.append((inp, b, d))
    return systems


@pytest.mark.parametrize("schedule", ["worklist", "chains"])
def test_batch_graph_matches_unbatched_and_oracle(schedule):
    import torch
    from paper_2607_05853_b300.api import batch_assemble, batch_release
    systems = _setup(SMALL)
    tuned = [b.autotune(with_projection=True) for _, b, _ in systems]
    assert all(t in (64, 96, 128, 160) for t, _ in tuned)
    assert all(p % 32 == 0 and 32 <= p <= 160 for _, p in tuned), tuned
    ref = [b.assemble() for _, b, _ in systems]
    torch.cuda.synchronize()
    Hs = [torch.zeros_like(r) for r in ref]
    stamps = batch_assemble([b for _, b, _ in systems], Hs, stamps=True, schedule=schedule)
    assert all(s > 0 for s in stamps)
    for (inp, b, _), H, R in zip(systems, Hs, ref):
        assert torch.equal(H, R), inp["name"]
        assert_split_close(H.cpu().numpy(), O.BSEOracle(inp).hamiltonian(), "bf16x3")
    for H in Hs:
        H.zero_()
    batch_assemble([b for _, b, _ in systems], Hs, schedule=schedule)   # replay of the cached graph
    torch.cuda.synchronize()
    for H, R in zip(Hs, ref):
        assert torch.equal(H, R)
    batch_release()


def test_batch_mixed_precisions():
    """An FP64 and a split context in the same graph (the chains schedule; the work list
    needs one split precision and refuses the pair)."""
    import torch
    from paper_2607_05853_b300.api import BseError, batch_assemble, batch_release
    a = _setup(SMALL[:1], "fp64")[0]
    b = _setup(SMALL[1:2], "bf16x2")[0]
    ra, rb = a[1].assemble(), b[1].assemble()
    Ha, Hb = torch.zeros_like(ra), torch.zeros_like(rb)
    with pytest.raises(BseError, match="EINVAL"):
        batch_assemble([a[1], b[1]], [Ha, Hb], schedule="worklist")
    batch_assemble([a[1], b[1]], [Ha, Hb], schedule="chains")
    torch.cuda.synchronize()
    assert torch.equal(Ha, ra) and torch.equal(Hb, rb)
    batch_release()


@pytest.mark.slow
@pytest.mark.parametrize("schedule", ["worklist", "chains"])
def test_sixteen_uneven_crystals_batch(schedule):
    """The 16-crystal batch (1-8 atoms, N_aux 86-579, meshes 6^3-10^3, Nv,Nc in {2,4,6}),
    complex64 split path, autotuned, one graph: per-system sampled blocks against the oracle
    for the smaller systems, exact equality with the unbatched assembly for all."""
    import torch
    from paper_2607_05853_b300.api import batch_assemble, batch_release
    specs = batched_specs(16)
    systems = _setup(specs)
    for _, b, _ in systems:
        b.autotune()
    Hs = [torch.empty((b.dim, b.dim), dtype=b.h_dtype, device="cuda") for _, b, _ in systems]
    stamps = batch_assemble([b for _, b, _ in systems], Hs, stamps=True, schedule=schedule)
    rng = np.random.default_rng(1)
    for (inp, b, _), H in zip(systems, Hs):
        ref = b.assemble()
        torch.cuda.synchronize()
        assert torch.equal(ref, H), inp["name"]
        del ref
        if b.naux <= 300:
            orc = O.BSEOracle(inp)
            n = orc.nvc
            # scale: the off-diagonal elements of a diagonal block (q = 0, the largest kernels)
            k0 = int(rng.integers(0, orc.nk))
            b0 = orc.block(k0, k0)
            scale = np.abs(b0 - np.diag(np.diag(b0))).max()
            worst = 0.0
            for _ in range(2):
                k1, k2 = (int(x) for x in rng.integers(0, orc.nk, 2))
                if k1 == k2:
                    continue
                blk = orc.block(k1, k2)
                got = H[k1 * n:(k1 + 1) * n, k2 * n:(k2 + 1) * n].cpu().numpy()
                worst, scale = max(worst, np.abs(got - blk).max()), max(scale, np.abs(blk).max())
            assert worst <= SAMPLED_OFF * scale, (inp["name"], worst / max(scale, 1e-300))
    print("batch stamps (ms):", [round(s / 1e6, 2) for s in stamps])
    batch_release()
