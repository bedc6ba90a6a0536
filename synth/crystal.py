"""Seeded synthetic crystals for the TDA-BSE hot path.

Every array produced here is an *input* of the method (the outputs of the DFT and GW
stages, steps 1-2 of the workflow in §III.B): band energies and coefficients on the
dense mesh (Eq. 2), LRI coefficients C^mu_st(R) (§III.A), the static screened
interaction W_mu,nu(R) on a Wigner-Seitz-folded coarse Born-von Karman cell (§III.B),
the truncated bare Coulomb matrix at q=0 (§III.A), and velocity matrix elements
<v k|v|c k> (Eq. abs_vel).

Recipe (seed = 20260000 + config unless given):
* tight binding h(R) for the R-set |R| <= r_max (lattice units), real Gaussian
  hoppings t0*N(0,1)*exp(-|R|/1.5) with h(-R) = h(R)^T, on-site split +-E_g/2 between
  the lower and upper halves of the orbitals; bands from numpy eigh per dense k;
* C^mu_st(R) = N(0,1)*exp(-d/2 Angstrom) for mu on the atom of s, else 0, with
  d = |tau_t + R - tau_s| (Cartesian);
* W(q_coarse) = s_W L(q) L(q)^dagger / N_aux with L(q) = sum_{|R'|<=1} G_R' e^{-2 pi i q.R'}
  e^{-|R'|}, G_R' real Gaussian, so that W(-q) = conj W(q) and W(R) is real; W(R) is
  the inverse transform on the coarse cell, each class copied to all of its
  minimal-length images with weight 1/(number of images);
* V0 = s_V L_V L_V^T / N_aux with L_V real Gaussian (symmetric positive semidefinite), and
  a bare V(R) on the R-set of W whose weighted sum is V0 (V(q) = V0 + a smooth PSD term
  that vanishes at q = 0);
* velocities from the tight-binding derivative sum_R i R_cart h(R) e^{2 pi i k.R}; the
  model itself (R_h, h_R, n_occ) is returned too, so that tests can rebuild h(k).

None of the method's own arithmetic (dense-mesh interpolation, pair projection, kernel
contraction, spectrum) is done here.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * np.pi


@dataclass
class CrystalSpec:
    name: str
    lattice: np.ndarray            # (3,3), rows are a_1,a_2,a_3 in Angstrom
    tau: np.ndarray                # (n_atoms,3) fractional positions
    nao: tuple                     # NAOs per atom
    naux: tuple                    # ABFs per atom
    coarse: tuple                  # coarse (GW) mesh
    dense: tuple                   # dense (BSE) mesh
    nv: int
    nc: int
    seed: int
    k_offset: tuple = (0.0, 0.0, 0.0)   # shift of the dense mesh, in units of its spacing
    r_max: float = 2.0             # radius of the h(R) and C(R) sets, lattice units
    two_d: bool = False
    e_gap: float = 6.0             # on-site split (eV)
    hop: float = 0.55              # hopping scale; t0 = hop / sqrt(N_ao)
    s_W: float = 0.04              # screened-interaction scale (eV); calibrated once on the
    s_V: float = 0.01              # tiny config so its singlet binding is ~0.13 eV, then frozen
    qp_shift: float = 0.5          # scissor on conduction bands (eV)

    @property
    def n_atoms(self):
        return len(self.nao)

    @property
    def n_ao(self):
        return int(sum(self.nao))

    @property
    def n_aux(self):
        return int(sum(self.naux))

    @property
    def n_k(self):
        return int(np.prod(self.dense))

    @property
    def dim(self):
        return self.n_k * self.nv * self.nc


def _fcc(a):
    h = a / 2.0
    return np.array([[0.0, h, h], [h, 0.0, h], [h, h, 0.0]])


def _hex(a, c):
    return np.array([[a, 0.0, 0.0], [-a / 2.0, a * np.sqrt(3.0) / 2.0, 0.0], [0.0, 0.0, c]])


def config_spec(i: int, seed: int | None = None) -> CrystalSpec:
    """The workloads: 0 tiny FP64, 1/2 FP64-at-scale (2 is the split-precision run on the
    same inputs), 4 differentiation monolayer.  Config 3 (16 uneven crystals) is
    produced by :func:`batched_specs`."""
    s = 20260000 + i if seed is None else seed
    diamond_tau = np.array([[0.0, 0.0, 0.0], [0.25, 0.25, 0.25]])
    if i == 0:
        return CrystalSpec("tiny-fp64", _fcc(5.43), diamond_tau, (4, 4), (20, 20),
                           (2, 2, 2), (4, 4, 4), 4, 4, s)
    if i in (1, 2):
        return CrystalSpec("fp64-at-scale" if i == 1 else "split-at-scale", _fcc(5.43),
                           diamond_tau, (13, 13), (75, 75), (4, 4, 4), (12, 12, 12), 4, 4,
                           20260001 if seed is None else seed)
    if i == 4:
        lat = _hex(3.19, 20.0)
        dz = 1.56 / 20.0
        tau = np.array([[0.0, 0.0, 0.0], [1 / 3, 2 / 3, dz], [2 / 3, 1 / 3, -dz]])
        return CrystalSpec("monolayer-grad", lat, tau, (15, 15, 15), (80, 80, 80),
                           (6, 6, 1), (30, 30, 1), 2, 2, s, two_d=True)
    raise ValueError(f"no single-crystal config {i}")


def scaled_spec(base: CrystalSpec, **kw) -> CrystalSpec:
    return dataclasses.replace(base, **kw)


def full_bse_spec(base: CrystalSpec) -> CrystalSpec:
    """The same crystal with the screened-interaction scale halved, for full-BSE workloads.

    The random band coefficients give conduction-valence products LRI coefficients as large
    as valence-valence ones, so the direct part of the coupling block is as large as that
    of the resonant block; at the calibrated s_W the matrix [[A, B], [B*, A*]] of config 0 is
    then indefinite (an unstable full BSE with complex excitation energies), at s_W / 2 it is
    positive definite with its lowest eigenvalue above 3 eV."""
    return dataclasses.replace(base, name=base.name + "-fullbse", s_W=base.s_W * 0.5)


def batched_specs(n: int = 16, seed: int = 20260003) -> list:
    """Config 3: n seeded crystals of uneven size (1-8 atoms, 9-13 NAOs/atom, 50-100
    ABFs/atom, dense meshes 6^3..10^3, Nv,Nc in {2,4,6}); coarse mesh ceil(dense/2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < n:
        na = int(rng.integers(1, 9))
        nao = tuple(int(x) for x in rng.integers(9, 14, size=na))
        naux = tuple(int(x) for x in rng.integers(50, 101, size=na))
        nd = int(rng.integers(6, 11))
        nv = int(rng.choice([2, 4, 6]))
        nc = int(rng.choice([2, 4, 6]))
        n_ao = sum(nao)
        if nv > n_ao // 2 or nc > n_ao - n_ao // 2:
            continue
        if rng.random() < 0.5:
            lat = np.eye(3) * (3.0 + 0.6 * na ** (1 / 3))
        else:
            lat = _hex(3.0 + 0.3 * na ** 0.5, 5.0 + 0.3 * na ** 0.5)
        tau = rng.random((na, 3))
        nc_mesh = (nd + 1) // 2
        out.append(CrystalSpec(f"batch{len(out)}", lat, tau, nao, naux,
                               (nc_mesh,) * 3, (nd,) * 3, nv, nc,
                               int(rng.integers(1, 2 ** 31)), r_max=1.5))
    return out


def r_set(r_max: float, two_d: bool) -> np.ndarray:
    n = int(np.floor(r_max))
    pts = []
    for a in range(-n, n + 1):
        for b in range(-n, n + 1):
            for c in ([0] if two_d else range(-n, n + 1)):
                if a * a + b * b + c * c <= r_max * r_max + 1e-9:
                    pts.append((a, b, c))
    pts.sort(key=lambda p: (p[0] ** 2 + p[1] ** 2 + p[2] ** 2, p))
    return np.array(pts, dtype=np.int32)


def kmesh_frac(mesh, offset=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Fractional k-points (n_i + offset_i)/N_i, flattened as (n1*N2 + n2)*N3 + n3."""
    n1, n2, n3 = mesh
    g = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1)
    g = g.reshape(-1, 3).astype(np.float64)
    return (g + np.asarray(offset, dtype=np.float64)) / np.asarray(mesh, dtype=np.float64)


def kmesh_index(mesh) -> np.ndarray:
    n1, n2, n3 = mesh
    g = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1)
    return g.reshape(-1, 3).astype(np.int64)


def _ws_images(coarse, lattice, two_d):
    """Minimal-length images of every coarse Born-von Karman class, weight 1/degeneracy."""
    cls = kmesh_index(coarse)
    reps, weights, owner = [], [], []
    N = np.asarray(coarse)
    rng3 = [0] if two_d else [-2, -1, 0, 1, 2]
    for ci, r0 in enumerate(cls):
        cands = []
        for m1 in (-2, -1, 0, 1, 2):
            for m2 in (-2, -1, 0, 1, 2):
                for m3 in rng3:
                    r = r0 + N * np.array([m1, m2, m3])
                    cands.append(r)
        cands = np.array(cands)
        ln = np.linalg.norm(cands @ lattice, axis=1)
        best = ln.min()
        sel = cands[ln <= best * (1 + 1e-9) + 1e-9]
        for r in sel:
            reps.append(r)
            weights.append(1.0 / len(sel))
            owner.append(ci)
    return np.array(reps, dtype=np.int32), np.array(weights), np.array(owner)


def make_inputs(spec: CrystalSpec, *, W_zero: bool = False, V_zero: bool = False) -> dict:
    """Generate every input array of one crystal (host numpy, float64/complex128)."""
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    lat = np.asarray(spec.lattice, dtype=np.float64)
    tau = np.asarray(spec.tau, dtype=np.float64)
    na, n_ao, n_aux = spec.n_atoms, spec.n_ao, spec.n_aux
    ao_atom = np.repeat(np.arange(na), spec.nao)
    aux_atom = np.repeat(np.arange(na), spec.naux)
    n_occ = n_ao // 2
    assert spec.nv <= n_occ and spec.nc <= n_ao - n_occ, "band window exceeds the basis"

    # ---- tight-binding model (input generator for Eq. 2's c and E) ----------------
    R_h = r_set(spec.r_max, spec.two_d)
    t0 = spec.hop / np.sqrt(n_ao)
    h = {}
    for R in R_h:
        key = tuple(int(x) for x in R)
        if key in h:
            continue
        mkey = tuple(-x for x in key)
        m = rng.standard_normal((n_ao, n_ao)) * t0 * np.exp(-np.linalg.norm(R) / 1.5)
        if key == (0, 0, 0):
            m = 0.5 * (m + m.T)
            h[key] = m
        else:
            h[key] = m
            h[mkey] = m.T.copy()
    # on-site split: the first n_occ orbitals in (local index, atom) order are "low"
    local = np.array([s - int(np.sum(spec.nao[: ao_atom[s]])) for s in range(n_ao)])
    order = sorted(range(n_ao), key=lambda s: (local[s], ao_atom[s]))
    onsite = np.full(n_ao, spec.e_gap / 2.0)
    onsite[order[:n_occ]] = -spec.e_gap / 2.0
    h[(0, 0, 0)] = h[(0, 0, 0)] + np.diag(onsite)
    hR = np.array([h[tuple(int(x) for x in R)] for R in R_h])

    kf = kmesh_frac(spec.dense, spec.k_offset)
    nk = kf.shape[0]
    ph = np.exp(1j * TWO_PI * (kf @ R_h.T.astype(np.float64)))          # [k, R]
    Hk = np.einsum("kr,rst->kst", ph, hR, optimize=True)
    Hk = 0.5 * (Hk + np.conj(np.transpose(Hk, (0, 2, 1))))
    E, U = np.linalg.eigh(Hk)
    vcols = [n_occ - 1 - v for v in range(spec.nv)]
    ccols = [n_occ + c for c in range(spec.nc)]
    cols = vcols + ccols
    c_k = np.ascontiguousarray(U[:, :, cols])
    e_ks = np.ascontiguousarray(E[:, cols])
    e_qp = e_ks.copy()
    e_qp[:, spec.nv:] += spec.qp_shift

    # velocity matrix elements <v k| dH/dk_alpha |c k>
    Rc = R_h.astype(np.float64) @ lat                                     # [R, 3] Cartesian
    vel = np.empty((3, nk, spec.nv, spec.nc), dtype=np.complex128)
    for a in range(3):
        dH = np.einsum("kr,rst->kst", ph * (1j * Rc[:, a])[None, :], hR, optimize=True)
        vel[a] = np.einsum("ksv,kst,ktc->kvc", np.conj(c_k[:, :, : spec.nv]), dH, c_k[:, :, spec.nv:], optimize=True)

    # ---- LRI coefficients C^mu_st(R), mu on the atom of s -----------------------
    R_C = r_set(spec.r_max, spec.two_d)
    C_R = np.zeros((len(R_C), n_ao, n_ao, n_aux))
    tau_c = tau @ lat
    for ir, R in enumerate(R_C):
        Rcart = R.astype(np.float64) @ lat
        d = np.linalg.norm(tau_c[None, :, :] + Rcart[None, None, :] - tau_c[:, None, :], axis=2)  # [A,B]
        for s in range(n_ao):
            A = ao_atom[s]
            mus = np.nonzero(aux_atom == A)[0]
            amp = np.exp(-d[A, ao_atom] / 2.0)                              # over t
            C_R[ir, s][:, mus] = rng.standard_normal((n_ao, len(mus))) * amp[:, None]

    # ---- screened interaction on the coarse mesh -> W(R) ---------------------------
    qc = kmesh_frac(spec.coarse)
    Rl = r_set(1.0, spec.two_d)
    G = rng.standard_normal((len(Rl), n_aux, n_aux))
    damp = np.exp(-np.linalg.norm(Rl, axis=1))
    Lq = np.einsum("qr,r,rmn->qmn", np.exp(-1j * TWO_PI * (qc @ Rl.T.astype(np.float64))), damp, G, optimize=True)
    Wq = spec.s_W * np.matmul(Lq, np.conj(np.transpose(Lq, (0, 2, 1)))) / n_aux
    R_W, w_RW, owner = _ws_images(spec.coarse, lat, spec.two_d)
    cls = kmesh_index(spec.coarse).astype(np.float64)
    Wcls = np.einsum("qc,qmn->cmn", np.exp(1j * TWO_PI * (qc @ cls.T)), Wq, optimize=True) / qc.shape[0]
    W_R = np.ascontiguousarray(Wcls.real[owner])
    LV = rng.standard_normal((n_aux, n_aux))
    V0 = spec.s_V * (LV @ LV.T) / n_aux
    # bare interaction on the coarse mesh: V(q) = V0 + s_V D(q) D(q)^dagger / N_aux with
    # D(q) = sum_{R' != 0} G'_R' (e^{-iq.R'} - 1) e^{-|R'|} (real G', so D(-q) = conj D(q) and
    # V(R) is real; D(0) = 0 keeps V(q = 0) = V0), folded to V(R) on the R-set of W.  Drawn
    # from a stream of its own, so the other inputs do not depend on it.
    rng_v = np.random.Generator(np.random.PCG64(spec.seed + 7919))
    Gv = rng_v.standard_normal((len(Rl), n_aux, n_aux))
    ph = np.exp(-1j * TWO_PI * (qc @ Rl.T.astype(np.float64))) - 1.0
    Dq = np.einsum("qr,r,rmn->qmn", ph, damp, Gv, optimize=True)
    Vq = V0[None] + spec.s_V * np.matmul(Dq, np.conj(np.transpose(Dq, (0, 2, 1)))) / n_aux
    Vcls = np.einsum("qc,qmn->cmn", np.exp(1j * TWO_PI * (qc @ cls.T)), Vq, optimize=True) / qc.shape[0]
    V_R = np.ascontiguousarray(Vcls.real[owner])
    if W_zero:
        W_R[:] = 0.0
        Wq[:] = 0.0
    if V_zero:
        V0[:] = 0.0
        V_R[:] = 0.0
        Vq[:] = 0.0

    return dict(
        name=spec.name, lattice=lat, tau=tau, volume=abs(np.linalg.det(lat)),
        nao=np.array(spec.nao, np.int32), naux=np.array(spec.naux, np.int32),
        ao_atom=ao_atom.astype(np.int32), aux_atom=aux_atom.astype(np.int32),
        dense=np.array(spec.dense, np.int32), coarse=np.array(spec.coarse, np.int32),
        k_offset=np.array(spec.k_offset, np.float64), kfrac=kf,
        nv=spec.nv, nc=spec.nc,
        R_C=R_C.astype(np.int32), C_R=C_R,
        R_W=R_W.astype(np.int32), w_RW=w_RW, W_R=W_R, W_q_coarse=Wq, q_coarse=qc,
        V0=V0, V_R=V_R, V_q_coarse=Vq, c_k=c_k, e_ks=e_ks, e_qp=e_qp, vel=vel,
        R_h=R_h.astype(np.int32), h_R=hR, n_occ=n_occ,
    )
