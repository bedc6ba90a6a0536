"""GPU parity of the FP64 path against the FP64 oracle (element by element), via the C ABI."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from synth import CrystalSpec, config_spec, make_inputs
from synth.crystal import _fcc, _hex

from helpers import gpu_hamiltonian, to_dev

pytestmark = pytest.mark.gpu

REL = 1e-10   # FP64 path: relative to max|H| (roughly 30 x FP64 eps x sqrt(summed terms))


@pytest.fixture(scope="module")
def cfg0():
    inp = make_inputs(config_spec(0))
    orc = O.BSEOracle(inp)
    return inp, orc, orc.hamiltonian()


def test_W_interpolation_matches_oracle(cfg0):
    inp, orc, _ = cfg0
    b, d, H, Wq = gpu_hamiltonian(inp, Wq=True)
    Wq = Wq.cpu().numpy()
    ref = np.stack([orc.W_q(iq) for iq in range(orc.nk)])
    assert np.abs(Wq - ref).max() <= REL * np.abs(ref).max()


def test_H_matches_oracle_elementwise(cfg0):
    inp, orc, Href = cfg0
    b, d, H, _ = gpu_hamiltonian(inp)
    H = H.cpu().numpy()
    scale = np.abs(Href).max()
    assert np.abs(H - Href).max() <= REL * scale
    assert np.abs(H - H.conj().T).max() <= 1e-13 * scale


@pytest.mark.parametrize("alpha", [0.0])
def test_triplet_matches_oracle(cfg0, alpha):
    inp, _, _ = cfg0
    ref = O.BSEOracle(inp, alpha=alpha).hamiltonian()
    b, d, H, _ = gpu_hamiltonian(inp, alpha=alpha)
    assert np.abs(H.cpu().numpy() - ref).max() <= REL * np.abs(ref).max()


RAGGED = {
    # nv != nc, odd mesh with an offset, N_aux not a multiple of anything, atoms of unequal size
    "ragged": CrystalSpec("ragged", _fcc(5.43), np.array([[0, 0, 0], [0.25, 0.25, 0.25]]), (3, 5), (17, 20),
                          (3, 1, 1), (3, 2, 5), 3, 2, 4242, k_offset=(0.5, 0.25, 0.1), r_max=1.5),
    # one atom, 1x1x1 mesh (brute-force-sized), single band pair
    "gamma_only": CrystalSpec("gamma", np.eye(3) * 4.0, np.zeros((1, 3)), (5,), (9,), (1, 1, 1), (1, 1, 1),
                              1, 1, 99, r_max=1.0),
    # 2-D monolayer-like: in-plane R only, three atoms
    "two_d": CrystalSpec("2d", _hex(3.19, 20.0), np.array([[0, 0, 0], [1 / 3, 2 / 3, 0.08], [2 / 3, 1 / 3, -0.08]]),
                         (3, 4, 3), (7, 6, 9), (2, 2, 1), (4, 3, 1), 2, 3, 1717, two_d=True),
    # window wider than the tile blocking: nv = nc = 6
    "wide": CrystalSpec("wide", _fcc(5.43), np.array([[0, 0, 0], [0.25, 0.25, 0.25]]), (7, 7), (11, 13),
                        (2, 1, 1), (2, 2, 2), 6, 6, 31337, r_max=1.0),
}


@pytest.mark.parametrize("name", list(RAGGED))
def test_ragged_shapes_match_oracle(name):
    inp = make_inputs(RAGGED[name])
    ref = O.BSEOracle(inp).hamiltonian()
    b, d, H, _ = gpu_hamiltonian(inp)
    assert np.abs(H.cpu().numpy() - ref).max() <= REL * np.abs(ref).max()


def test_dipole_vector(cfg0):
    inp, orc, _ = cfg0
    b, d, H, _ = gpu_hamiltonian(inp)
    u = b.dipole_vector(d["vel"], d["e_ks"])
    b.sync()
    assert np.allclose(u.cpu().numpy(), np.conj(orc.dipoles()), rtol=1e-13, atol=0)


def test_spectrum_full_length_equals_exact(cfg0):
    import torch
    inp, orc, Href = cfg0
    b, d, H, _ = gpu_hamiltonian(inp)
    u = b.dipole_vector(d["vel"], d["e_ks"])
    om = torch.linspace(0, 10, 401, dtype=torch.float64, device="cuda")
    eps = b.spectrum(H, u, b.dim, om, 0.1, orc.prefactor())
    b.sync()
    ref = O.eps2_exact(Href, orc.dipoles(), om.cpu().numpy(), 0.1, orc.prefactor())
    assert np.abs(eps.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()


def test_haydock_coefficients_match_oracle(cfg0):
    import torch
    inp, orc, Href = cfg0
    b, d, H, _ = gpu_hamiltonian(inp)
    u = b.dipole_vector(d["vel"], d["e_ks"])
    n = 120
    ab = torch.empty((3, 3, n), dtype=torch.float64, device="cuda")
    om = torch.linspace(0, 10, 101, dtype=torch.float64, device="cuda")
    eps = b.spectrum(H, u, n, om, 0.1, orc.prefactor(), ab=ab)
    b.sync()
    ab = ab.cpu().numpy()
    ref_eps = np.zeros(101)
    for p in range(3):
        a, bb, b0 = O.haydock_coeffs(Href, np.conj(orc.dipoles()[p]), n)
        assert np.allclose(ab[p, 0, :len(a)], a, rtol=0, atol=1e-10 * np.abs(a).max())
        assert np.allclose(ab[p, 1, :len(bb)], bb, rtol=0, atol=1e-10 * np.abs(a).max())
        assert np.isclose(ab[p, 2, 0], b0, rtol=1e-13)
        ref_eps += orc.prefactor() * O.haydock_eps2(a, bb, b0, om.cpu().numpy(), 0.1)
    assert np.abs(eps.cpu().numpy() - ref_eps).max() <= 1e-9 * np.abs(ref_eps).max()


def test_lowest_excitons_match_lapack(cfg0):
    inp, orc, Href = cfg0
    b, d, H, _ = gpu_hamiltonian(inp)
    om, rs = b.lowest(H, 10, 400)
    b.sync()
    ref = np.linalg.eigvalsh(Href)[:10]
    om, rs = om.cpu().numpy(), rs.cpu().numpy()
    conv = rs < 1e-8
    assert conv[:4].all()
    assert np.all(np.abs(om[conv] - ref[conv]) <= rs[conv] + 1e-10)


def test_out_of_order_and_bad_pointers():
    from paper_2607_05853_b300.api import BSE, BseError
    inp = make_inputs(config_spec(0))
    b = BSE.from_inputs(inp)
    with pytest.raises(BseError, match="ESTATE"):
        b.assemble()
    d = to_dev(inp)
    with pytest.raises(BseError, match="ESTATE"):
        b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
    b.close()


@pytest.mark.slow
def test_full_size_fp64_sampled_blocks():
    """The FP64-at-scale workload (27648 x 27648, 1728 k, N_aux 150): the whole matrix is
    built on the device and a seeded sample of blocks (including q = 0 and the last row
    and column) is compared with the oracle block by block."""
    inp = make_inputs(config_spec(1))
    b, d, H, _ = gpu_hamiltonian(inp)
    orc = O.BSEOracle(inp)
    rng = np.random.default_rng(11)
    nk, n = orc.nk, orc.nvc
    pairs = [(0, 0), (nk - 1, nk - 1), (0, nk - 1), (nk - 1, 0)] + [tuple(rng.integers(0, nk, 2)) for _ in range(12)]
    scale = 0.0
    worst = 0.0
    for k1, k2 in pairs:
        ref = orc.block(int(k1), int(k2))
        got = H[k1 * n:(k1 + 1) * n, k2 * n:(k2 + 1) * n].cpu().numpy()
        scale = max(scale, np.abs(ref).max())
        worst = max(worst, np.abs(got - ref).max())
    assert worst <= REL * scale
    # Hermiticity of the whole device matrix, sampled by rows
    for r in rng.integers(0, b.dim, 8):
        row = H[int(r), :].cpu().numpy()
        col = H[:, int(r)].cpu().numpy()
        assert np.abs(row - np.conj(col)).max() <= 1e-12 * scale


@pytest.mark.parametrize("name", ["tiny", "two_d"])
def test_interp_V_matches_oracle(name):
    """bse_interp_V: the bare V(q) at every dense q against the oracle's R-sum (FP64), for an
    FP64 and a split-precision context; V(q = 0) is the V(0) of the exchange."""
    import torch
    from paper_2607_05853_b300.api import BSE
    inp = make_inputs(config_spec(0) if name == "tiny" else RAGGED[name])
    n1, n2, n3 = (int(x) for x in inp["dense"])
    nk = n1 * n2 * n3
    for prec in ("fp64", "bf16x3"):
        b = BSE.from_inputs(inp, precision=prec)
        Vq = b.interp_V(torch.from_numpy(np.ascontiguousarray(inp["V_R"])).cuda()).cpu().numpy()
        b.sync()
        scale = np.abs(inp["V0"]).max()
        for q in range(nk):
            qf = np.array([q // (n2 * n3), (q // n3) % n2, q % n3], np.float64) / np.array([n1, n2, n3])
            ref = O.interp_V(inp["V_R"], inp["R_W"], inp["w_RW"], qf)
            assert np.abs(Vq[q] - ref).max() <= 1e-12 * scale, (prec, q)
        assert np.abs(Vq[0] - inp["V0"]).max() <= 1e-12 * scale
