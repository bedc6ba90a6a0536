"""Plain FP64 oracle of the Tamm-Dancoff BSE hot path (numpy, CPU) -- test infrastructure.

What it computes, and where each step comes from in the paper (arXiv 2607.05853):

* W_mu,nu(q) = sum_R w_R W_mu,nu(R) exp(-i q.R) with q = k1 - k2: the R-sum inside
  Eq. W_LRI (§III.A), whose phase is exp(i(k2-k1).R); w_R are the weights of the
  Wigner-Seitz images of the coarse Born-von Karman cell (§III.B).
* C^mu_st(k) = sum_R C^mu_st(R) exp(+i k.R), with C^mu_st nonzero only for mu on the
  atom of s (the two-centre expansion and its Fourier transform, §III.A).
* C~^mu_{j k2, i k1} = sum_st conj(c^{k2}_sj) c^{k1}_ti [C^mu_st(k1) + C^mu_ts(-k2)]
  (the Kohn-Sham-basis LRI coefficients, §III.A).
* direct kernel (j k2*, i k1|W|a k1*, b k2) = (1/N_k) sum_mu,nu C~^mu_{j k2,i k1}
  W_mu,nu(k1-k2) C~^nu_{a k1,b k2} (Eq. W_LRI) and exchange kernel
  (a k1*, i k1|V|j k2*, b k2) = (1/N_k) sum C~^mu_{a k1,i k1} V_mu,nu(0) C~^nu_{j k2,b k2}.
* A_{ai k1, bj k2} = (E^GW_a k1 - E^GW_i k1) delta + alpha * exchange - direct
  (Eq. Hamiltonian, §II.C; alpha = 2 singlet, 0 triplet).
* eps2(omega) = 4 pi^2/(3 N_k V) sum_S |sum_{aik} <ik|v|ak>/(E_ak - E_ik) X^S_aik|^2
  delta(omega - Omega_S) (Eq. abs_vel), the delta broadened to a Lorentzian of
  half-width eta; the exact sum uses a LAPACK eigendecomposition, and a plain Haydock
  (Lanczos) recursion gives the same quantity through a continued fraction.
* lowest exciton energies: LAPACK eigvalsh of the Hermitian TDA matrix.
* the windowed absorption integral I = int_lo^hi eps2(omega) domega (eps2 as above) and
  its seed Gamma with dI = tr(Gamma dH), by the Daleckii-Krein formula for the derivative
  of a matrix function on the full eigendecomposition.
* full BSE (§II.C): the coupling block B_{ai k1, bj k2} = alpha (a k1*, i k1|V|b k2*, j k2)
  - (b k2*, i k1|W|a k1*, j k2) with both kernels in the LRI form of Eq. W_LRI
  ((1/N_k) C~ V(0) C~ and (1/N_k) C~^mu_{b k2, i k1} W(k1-k2) C~^nu_{a k1, j k2}); the
  Hamiltonian [[A, B], [-B*, -A*]]; its paired solutions +-Omega with right eigenvectors
  (X, Y), normalised X^dagger X - Y^dagger Y = 1, found by the structure-preserving route
  (the Hermitian positive definite M = [[A, B], [B*, A*]] made real by a unitary change of
  basis, its Cholesky factor L, and the Hermitian eigenproblem of L^T K L, K the image of
  diag(1, -1)); and eps2 with the Y term (Eq. full_BSE_epsilon2): the amplitude
  sum d X - conj(d) Y, since <ak|v|ik> = conj(<ik|v|ak>) and E_i - E_a = -(E_a - E_i).
* finite exciton momentum Q (the q != 0 extension the paper names as future work, §V):
  the pair (k, i, a) holds the valence band i at k and the conduction band a at k + Q, so
  every conduction coefficient, LRI coefficient and energy of the pair is taken at k + Q.
  The same C~ definition (§III.A) and kernel forms (Eq. W_LRI) apply: the direct kernel
  keeps W at q = k1 - k2 (both conduction points shift by Q), the diagonal is
  E_a(k+Q) - E_i(k), and the exchange densities psi*_{a k+Q} psi_{i k} and
  psi*_{j k2} psi_{b k2+Q} expand in ABF Bloch sums of momentum -Q and +Q, whose Coulomb
  integral over the crystal is N_k sum_R w_R Vbar(R) e^{+i Q.R} = N_k V(-Q) in the
  convention V(q) = sum_R w_R Vbar(R) e^{-i q.R}.  At Q = 0 this is V(0) and the TDA
  Hamiltonian above.

Index conventions: the H row of (k, v, c) is (k*Nv + v)*Nc + c; valence window column
v=0 is the valence band maximum (counting down), conduction column c=0 the conduction
band minimum (counting up); k is flattened (n1*N2 + n2)*N3 + n3.

Everything is FP64 / complex128, evaluated element block by element block from the
definitions above; W(q) per q and C(k) per k are memoised (this does not change what
is computed).  Nothing here is shared with, or imported from, the CUDA path.

Pins (tests/test_oracle_pins.py) tie every function to something outside it: a real-space
brute force of both kernels (A, B, finite Q), FFT and coarse-mesh identities of the
interpolation, LAPACK, closed forms of the spectrum and of the full BSE, sum rules, central
differences of the gradients, and for the dipoles the overlaps <i|d a/dk> from finite
differences of the tight-binding eigenvectors.  Parity unpinned: the spin factor inside
spectrum_prefactor (a reading of the paper's normalisation, shared by both sides) and
absolute values against the paper's tables (its inputs are not available).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "interp_W", "lri_C_k", "ks_lri", "BSEOracle", "eps2_exact", "haydock_coeffs",
    "haydock_eps2", "lowest_excitons", "spectrum_prefactor", "binding_energy",
    "adjoint_seed_lowest", "grad_from_seed", "window_weight", "window_integral", "window_seed_exact", "offset_average_eps2", "interp_V",
    "full_hamiltonian", "full_bse_pairs", "eps2_full_exact",
]

TWO_PI = 2.0 * np.pi


def interp_W(W_R, R_W, w_RW, q):
    """W_mu,nu(q) = sum_R w_R W_mu,nu(R) e^{-i q.R}; q fractional (Eq. W_LRI's R-sum)."""
    ph = np.exp(-1j * TWO_PI * (np.asarray(R_W, np.float64) @ np.asarray(q, np.float64)))
    return np.einsum("r,rmn->mn", ph * np.asarray(w_RW), W_R)


def lri_C_k(C_R, R_C, k, ao_atom, aux_atom):
    """C^mu_st(k) = sum_R C^mu_st(R) e^{+i k.R} for mu on the atom of s, else 0 (§III.A).

    Returns an array indexed [s, t, mu]."""
    ph = np.exp(1j * TWO_PI * (np.asarray(R_C, np.float64) @ np.asarray(k, np.float64)))
    Ck = np.einsum("r,rstu->stu", ph, C_R)
    own = (np.asarray(ao_atom)[:, None] == np.asarray(aux_atom)[None, :])   # [s, mu]
    return Ck * own[:, None, :]


def ks_lri(c_bra, c_ket, C_of_kket, C_of_minus_kbra):
    """C~^mu_{m k', n k} = sum_st conj(c^{k'}_sm) c^k_tn [C^mu_st(k) + C^mu_ts(-k')] (§III.A).

    c_bra = c^{k'} [s, m], c_ket = c^k [t, n]; C_of_kket = C(k) [s,t,mu];
    C_of_minus_kbra = C(-k') [s,t,mu].  Returns [mu, m, n]."""
    t1 = np.einsum("sm,tn,stu->umn", np.conj(c_bra), c_ket, C_of_kket, optimize=True)
    t2 = np.einsum("sm,tn,tsu->umn", np.conj(c_bra), c_ket, C_of_minus_kbra, optimize=True)
    return t1 + t2


class BSEOracle:
    """Element-block evaluation of the TDA Hamiltonian A from the definitions above."""

    def __init__(self, inp: dict, alpha: float = 2.0, Q=(0, 0, 0)):
        """Q: exciton momentum in dense-mesh steps (Q_frac = Q / N per axis).  Q != 0 with
        alpha != 0 needs inp["V_R"] (the exchange takes V(-Q) from the R-sum)."""
        self.inp = inp
        self.alpha = float(alpha)
        self.mesh = np.asarray(inp["dense"], np.int64)
        self.nk = int(np.prod(self.mesh))
        self.nv, self.nc = int(inp["nv"]), int(inp["nc"])
        self.nvc = self.nv * self.nc
        self.dim = self.nk * self.nvc
        n1, n2, n3 = self.mesh
        g = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1)
        self.kint = g.reshape(-1, 3)
        self.kfrac = (self.kint + np.asarray(inp["k_offset"], np.float64)) / self.mesh
        self.Q = np.mod(np.asarray(Q, np.int64), self.mesh)
        self.finite_Q = bool(np.any(self.Q != 0))
        if not self.finite_Q:
            self.V_exch = inp["V0"]
        elif self.alpha != 0.0:
            self.V_exch = interp_V(inp["V_R"], inp["R_W"], inp["w_RW"], -self.Q / self.mesh)
        else:
            self.V_exch = None
        self._Ck, self._Cmk, self._Wq, self._X1, self._X2 = {}, {}, {}, {}, {}

    # -- memoised pieces ---------------------------------------------------------
    def C_k(self, ik):
        if ik not in self._Ck:
            i = self.inp
            self._Ck[ik] = lri_C_k(i["C_R"], i["R_C"], self.kfrac[ik], i["ao_atom"], i["aux_atom"])
        return self._Ck[ik]

    def C_mk(self, ik):
        if ik not in self._Cmk:
            i = self.inp
            self._Cmk[ik] = lri_C_k(i["C_R"], i["R_C"], -self.kfrac[ik], i["ao_atom"], i["aux_atom"])
        return self._Cmk[ik]

    def kQ(self, ik):
        """Mesh index of k + Q (the conduction point of the pairs at k)."""
        d = np.mod(self.kint[ik] + self.Q, self.mesh)
        return int((d[0] * self.mesh[1] + d[1]) * self.mesh[2] + d[2])

    def q_index(self, ik1, ik2):
        d = np.mod(self.kint[ik1] - self.kint[ik2], self.mesh)
        return int((d[0] * self.mesh[1] + d[1]) * self.mesh[2] + d[2])

    def W_q(self, iq):
        if iq not in self._Wq:
            i = self.inp
            n1, n2, n3 = self.mesh
            qv = np.array([iq // (n2 * n3), (iq // n3) % n2, iq % n3], np.float64) / self.mesh
            self._Wq[iq] = interp_W(i["W_R"], i["R_W"], i["w_RW"], qv)
        return self._Wq[iq]

    def _cv(self, ik):
        return self.inp["c_k"][ik][:, : self.nv]

    def _cc(self, ik):
        return self.inp["c_k"][ik][:, self.nv:]

    def X_exch_left(self, ik):       # C~^mu_{a k+Q, i k}  -> [mu, a, i]
        if ik not in self._X1:
            kq = self.kQ(ik)
            self._X1[ik] = ks_lri(self._cc(kq), self._cv(ik), self.C_k(ik), self.C_mk(kq))
        return self._X1[ik]

    def X_exch_right(self, ik):      # C~^nu_{j k, b k+Q}  -> [nu, j, b]
        if ik not in self._X2:
            kq = self.kQ(ik)
            self._X2[ik] = ks_lri(self._cv(ik), self._cc(kq), self.C_k(kq), self.C_mk(ik))
        return self._X2[ik]

    def M_vv(self, ik1, ik2):        # C~^mu_{j k2, i k1} -> [mu, j, i]
        return ks_lri(self._cv(ik2), self._cv(ik1), self.C_k(ik1), self.C_mk(ik2))

    def M_cc(self, ik1, ik2):        # C~^nu_{a k1+Q, b k2+Q} -> [nu, a, b]
        p1, p2 = self.kQ(ik1), self.kQ(ik2)
        return ks_lri(self._cc(p1), self._cc(p2), self.C_k(p2), self.C_mk(p1))

    # -- kernels and blocks ------------------------------------------------------------
    def direct(self, ik1, ik2):
        """(j k2*, i k1|W|a k1*, b k2) as [i, a, j, b] (Eq. W_LRI)."""
        Wq = self.W_q(self.q_index(ik1, ik2))
        Mv, Mc = self.M_vv(ik1, ik2), self.M_cc(ik1, ik2)
        T = np.einsum("uji,uv->jiv", Mv, Wq)
        return np.einsum("jiv,vab->iajb", T, Mc) / self.nk

    def exchange(self, ik1, ik2):
        """(a k1+Q*, i k1|V|j k2*, b k2+Q) as [i, a, j, b] (the V-kernel beside Eq. W_LRI;
        V(0) at Q = 0, V(-Q) otherwise)."""
        X1, X2 = self.X_exch_left(ik1), self.X_exch_right(ik2)
        T = np.einsum("uai,uv->aiv", X1, self.V_exch)
        return np.einsum("aiv,vjb->iajb", T, X2) / self.nk

    def block(self, ik1, ik2):
        """H block of rows (k1, i, a) and columns (k2, j, b), shape (Nv*Nc, Nv*Nc) (Eq. Hamiltonian)."""
        blk = -self.direct(ik1, ik2)
        if self.alpha != 0.0:
            blk = blk + self.alpha * self.exchange(ik1, ik2)
        blk = blk.reshape(self.nvc, self.nvc)
        if ik1 == ik2:
            ev, ec = self.inp["e_qp"][ik1][: self.nv], self.inp["e_qp"][self.kQ(ik1)][self.nv:]
            de = (ec[None, :] - ev[:, None]).reshape(-1)                     # (i, a)
            blk = blk + np.diag(de)
        return blk

    # -- coupling block of the full BSE (§II.C) -------------------------------------------
    def coupling_exchange(self, ik1, ik2):
        """(a k1*, i k1|V|b k2*, j k2) as [i, a, j, b]: C~_{a k1, i k1} V(0) C~_{b k2, j k2} / N_k."""
        X1, X2 = self.X_exch_left(ik1), self.X_exch_left(ik2)          # [mu, a, i], [nu, b, j]
        return np.einsum("uai,uv,vbj->iajb", X1, self.V_exch, X2, optimize=True) / self.nk

    def coupling_direct(self, ik1, ik2):
        """(b k2*, i k1|W|a k1*, j k2) as [i, a, j, b]: C~_{b k2, i k1} W(k1-k2) C~_{a k1, j k2} / N_k."""
        Wq = self.W_q(self.q_index(ik1, ik2))
        M1 = ks_lri(self._cc(ik2), self._cv(ik1), self.C_k(ik1), self.C_mk(ik2))   # [mu, b, i]
        M2 = ks_lri(self._cc(ik1), self._cv(ik2), self.C_k(ik2), self.C_mk(ik1))   # [nu, a, j]
        return np.einsum("ubi,uv,vaj->iajb", M1, Wq, M2, optimize=True) / self.nk

    def coupling_block(self, ik1, ik2):
        blk = -self.coupling_direct(ik1, ik2)
        if self.alpha != 0.0:
            blk = blk + self.alpha * self.coupling_exchange(ik1, ik2)
        return blk.reshape(self.nvc, self.nvc)

    def coupling(self):
        """B of Eq. Hamiltonian, [dim, dim] (rows (k1, i, a), columns (k2, j, b)); Q = 0 only."""
        if self.finite_Q:
            raise ValueError("coupling: the full BSE is built at Q = 0")
        B = np.empty((self.dim, self.dim), np.complex128)
        n = self.nvc
        for k1 in range(self.nk):
            for k2 in range(self.nk):
                B[k1 * n:(k1 + 1) * n, k2 * n:(k2 + 1) * n] = self.coupling_block(k1, k2)
        return B

    def hamiltonian(self):
        H = np.empty((self.dim, self.dim), np.complex128)
        n = self.nvc
        for k1 in range(self.nk):
            for k2 in range(self.nk):
                H[k1 * n:(k1 + 1) * n, k2 * n:(k2 + 1) * n] = self.block(k1, k2)
        return H

    # -- optics ------------------------------------------------------------------------
    def dipoles(self):
        """d_alpha,(k,i,a) = <ik|v_alpha|ak>/(E^KS_ak - E^KS_ik) (Eq. abs_vel), shape [3, dim].
        Optical (vertical) transitions only: defined at Q = 0."""
        if self.finite_Q:
            raise ValueError("dipoles: the optical matrix elements are vertical (Q = 0)")
        e = self.inp["e_ks"]
        de = e[:, self.nv:][:, None, :] - e[:, : self.nv][:, :, None]        # [k, i, a]
        return (self.inp["vel"] / de[None]).reshape(3, -1)

    def prefactor(self):
        return spectrum_prefactor(self.nk, float(self.inp["volume"]))


def full_hamiltonian(A, B):
    """The full BSE matrix [[A, B], [-B*, -A*]] (§II.C)."""
    return np.block([[A, B], [-np.conj(B), -np.conj(A)]])


def full_bse_pairs(A, B):
    """Positive solutions Omega_S of the full BSE with right eigenvectors (X_S, Y_S) normalised
    X^dagger X - Y^dagger Y = 1 (the paired formulation of §II.C).

    M = [[A, B], [B*, A*]] is Hermitian positive definite for a stable excited state.  With
    U = (1/sqrt 2) [[1, -i], [1, i]] (blocks of identities) U^dagger M U = M_r is real
    symmetric and U^dagger diag(1, -1) U = K = [[0, -i], [i, 0]], so H = diag(1,-1) M becomes
    K M_r.  With M_r = L L^T, the Hermitian matrix S = L^T K L has the eigenvalues of H; an
    orthonormal eigenvector w of S gives z = L^-T w with z^T M_r z = 1 and the eigenvector
    Z = U z of H with Z^dagger M Z = 1; for Omega > 0, sqrt(Omega) Z = (X, Y) has
    X^dagger X - Y^dagger Y = Z^dagger diag(1,-1) Z Omega = 1.
    Returns (Omega [n] ascending, X [dim, n], Y [dim, n])."""
    n = A.shape[0]
    I = np.eye(n)
    M = np.block([[A, B], [np.conj(B), np.conj(A)]])
    U = np.block([[I, -1j * I], [I, 1j * I]]) / np.sqrt(2.0)
    Mr = U.conj().T @ M @ U
    if np.abs(Mr.imag).max() > 1e-10 * max(np.abs(Mr).max(), 1e-300):
        raise ValueError("full_bse_pairs: [[A, B], [B*, A*]] lacks the expected structure")
    L = np.linalg.cholesky(0.5 * (Mr.real + Mr.real.T))
    K = np.block([[np.zeros((n, n)), -1j * I], [1j * I, np.zeros((n, n))]])
    S = L.T @ K @ L
    lam, Wv = np.linalg.eigh(0.5 * (S + S.conj().T))
    pos = lam > 0
    z = np.linalg.solve(L.T, Wv[:, pos])
    Z = (U @ z) * np.sqrt(lam[pos])[None, :]
    return lam[pos], Z[:n], Z[n:]


def eps2_full_exact(A, B, d, omega, eta, pref):
    """Full-BSE eps2 (Eq. full_BSE_epsilon2) with a Lorentzian of half width eta:
    pref sum_S |sum_r d_r X_rS - conj(d_r) Y_rS|^2 L(omega - Omega_S), per polarisation summed."""
    w, X, Y = full_bse_pairs(A, B)
    d = np.atleast_2d(np.asarray(d))
    osc = np.abs(d @ X - np.conj(d) @ Y) ** 2                              # [pol, S]
    L = (eta / np.pi) / ((np.asarray(omega)[:, None] - w[None, :]) ** 2 + eta ** 2)
    return pref * (L @ osc.sum(axis=0))


def spectrum_prefactor(nk, volume):
    """4 pi^2 / (3 N_k V) of Eq. abs_vel (spin factor 1: the 1/sqrt2 normalisation and the
    spin sum of the singlet cancel)."""
    return 4.0 * np.pi ** 2 / (3.0 * nk * volume)


def eps2_exact(H, d, omega, eta, pref):
    """Eq. abs_vel with a Lorentzian of half-width eta, from a full eigendecomposition."""
    w, X = np.linalg.eigh(H)
    osc = np.abs(np.asarray(d) @ X) ** 2                                   # [pol, S]
    L = (eta / np.pi) / ((np.asarray(omega)[:, None] - w[None, :]) ** 2 + eta ** 2)
    return pref * (L @ osc.sum(axis=0))


def haydock_coeffs(H, u, n_steps, reorth=True):
    """Lanczos recursion on (H, u): returns (a[1..n], b[1..n], ||u||).

    q_1 = u/||u||; w = H q_j - a_j q_j - b_{j-1} q_{j-1}, a_j = q_j^H H q_j,
    b_j = ||w|| after (optional, twice-applied) full reorthogonalisation; stops early if
    b_j < 1e-14 * ||H||_max."""
    u = np.asarray(u, np.complex128)
    beta0 = np.linalg.norm(u)
    n = H.shape[0]
    Q = np.zeros((n_steps + 1, n), np.complex128)
    a = np.zeros(n_steps)
    b = np.zeros(n_steps)
    Q[0] = u / beta0
    hmax = np.abs(H).max()
    prev = np.zeros(n, np.complex128)
    bprev = 0.0
    m = n_steps
    for j in range(n_steps):
        w = H @ Q[j]
        a[j] = np.vdot(Q[j], w).real
        w = w - a[j] * Q[j] - bprev * prev
        if reorth:
            for _ in range(2):
                w = w - Q[: j + 1].T @ (np.conj(Q[: j + 1]) @ w)
        b[j] = np.linalg.norm(w)
        if j == n_steps - 1:
            break
        if b[j] < 1e-14 * hmax:
            m = j + 1
            break
        prev, bprev = Q[j], b[j]
        Q[j + 1] = w / b[j]
    return a[:m], b[:m], beta0


def haydock_eps2(a, b, beta0, omega, eta):
    """-(1/pi) Im g(omega + i eta), g(z) = beta0^2/(z - a1 - b1^2/(z - a2 - ...))."""
    z = np.asarray(omega, np.float64) + 1j * eta
    f = z - a[-1]
    for j in range(len(a) - 2, -1, -1):
        f = z - a[j] - b[j] ** 2 / f
    return -(beta0 ** 2 / f).imag / np.pi


def lowest_excitons(H, n):
    """Lowest n eigenvalues of the Hermitian TDA matrix (LAPACK)."""
    return np.linalg.eigvalsh(H)[:n]


def binding_energy(e_qp, nv, omega1):
    """E_B = min_k (E^QP_ck - E^QP_vk) - Omega_1 over the band edges (§IV, exciton binding)."""
    return float(np.min(e_qp[:, nv] - e_qp[:, 0]) - omega1)


# ---------------------------------------------------------------------------- gradients
def adjoint_seed_lowest(H, n):
    """Eigenpairs (Omega_S, x_S) of the n lowest excitons and the Hellmann-Feynman seeds
    Gamma_S = x_S x_S^dagger, so that dOmega_S = tr(Gamma_S dH) for a Hermitian dH."""
    w, X = np.linalg.eigh(H)
    return w[:n], X[:, :n]


def grad_from_seed(orc, Gamma):
    """dL/dW(R) and dL/dE^QP for dL = tr(Gamma dH) (Gamma Hermitian, e.g. x x^dagger).

    H depends on W only through the direct term -(1/N_k) sum M_vv W(q) M_cc (Eq. W_LRI), with
    W(q) = sum_R w_R W(R) e^{-i q.R}; the gradient with respect to one real entry W_mu,nu(R)
    is Re tr(Gamma dH/dW_mu,nu(R)) (the symmetric pair W_mu,nu(R), W_nu,mu(-R) together moves
    the energy by twice this).  E^QP enters only the diagonal (Eq. Hamiltonian):
    dL/dE^QP_a,k+Q = sum_i Gamma_(k,i,a),(k,i,a), dL/dE^QP_ik = -sum_a Gamma_(k,i,a),(k,i,a).
    Returns (dW_R [n_RW][N_aux][N_aux], de_qp [N_k][Nv+Nc])."""
    inp = orc.inp
    nk, nv, nc, nvc = orc.nk, orc.nv, orc.nc, orc.nvc
    naux = inp["W_R"].shape[1]
    Aq = np.zeros((nk, naux, naux), np.complex128)
    for k1 in range(nk):
        for k2 in range(nk):
            iq = orc.q_index(k1, k2)
            Mv, Mc = orc.M_vv(k1, k2), orc.M_cc(k1, k2)          # [mu, j, i], [nu, a, b]
            # Gamma block with rows (k2, j, b) and columns (k1, i, a)
            G = Gamma[k2 * nvc:(k2 + 1) * nvc, k1 * nvc:(k1 + 1) * nvc].reshape(nv, nc, nv, nc)  # [j,b,i,a]
            Aq[iq] += -np.einsum("uji,jbia,vab->uv", Mv, G, Mc, optimize=True) / nk
    # adjoint of W(q) = sum_R w_R W(R) e^{-i q.R}
    n1, n2, n3 = orc.mesh
    qint = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1).reshape(-1, 3)
    qfrac = qint / orc.mesh
    ph = np.exp(-1j * TWO_PI * (qfrac @ inp["R_W"].astype(np.float64).T))            # [q, R]
    dW = np.real(np.einsum("qr,quv->ruv", ph, Aq)) * inp["w_RW"][:, None, None]
    d = np.real(np.diag(Gamma)).reshape(nk, nv, nc)
    de = np.zeros((nk, nv + nc))
    for k in range(nk):                  # the conduction energy of the pairs at k sits at k + Q
        de[orc.kQ(k), nv:] += d[k].sum(axis=0)
    de[:, :nv] = -d.sum(axis=2)
    return dW, de


def window_weight(x, lo, hi, eta):
    """f(x) = int_lo^hi (1/pi) eta / ((omega - x)^2 + eta^2) domega: the Lorentzian of
    Eq. abs_vel (half width eta) integrated over the window [lo, hi]."""
    x = np.asarray(x, dtype=np.float64)
    return (np.arctan((hi - x) / eta) - np.arctan((lo - x) / eta)) / np.pi


def window_integral(H, d, lo, hi, eta, pref):
    """I = int_lo^hi eps2(omega) domega for eps2 of Eq. abs_vel (Lorentzian half width eta),
    from a full eigendecomposition: pref sum_S |sum_r d_r X_rS|^2 f(Omega_S)."""
    w, X = np.linalg.eigh(H)
    osc = np.abs(np.asarray(d) @ X) ** 2
    return pref * float(osc.sum(axis=0) @ window_weight(w, lo, hi, eta))


def window_seed_exact(H, d, lo, hi, eta, pref):
    """Gamma with dI = tr(Gamma dH) for the window integral I, from the Daleckii-Krein
    derivative of the matrix function f(H): with H = X diag(w) X^dagger,
    df(H) = X (F o (X^dagger dH X)) X^dagger, F_ST = (f(w_S) - f(w_T)) / (w_S - w_T)
    (f'(w_S) where w_S = w_T).  I = pref sum_p u_p^dagger f(H) u_p with u_p = conj(d_p)
    gives Gamma = pref sum_p X (F o c_p c_p^dagger) X^dagger, c_p = X^dagger u_p."""
    w, X = np.linalg.eigh(H)
    f = window_weight(w, lo, hi, eta)
    ya, yb = lo - w, hi - w
    df = (eta / (ya ** 2 + eta ** 2) - eta / (yb ** 2 + eta ** 2)) / np.pi
    gap = w[:, None] - w[None, :]
    close = np.abs(gap) <= 1e-9 * (np.abs(w[:, None]) + np.abs(w[None, :]) + eta)
    F = np.where(close, 0.5 * (df[:, None] + df[None, :]), (f[:, None] - f[None, :]) / np.where(close, 1.0, gap))
    G = np.zeros(H.shape, np.complex128)
    for dp in np.asarray(d):
        c = X.conj().T @ np.conj(dp)
        G += X @ (F * np.outer(c, c.conj())) @ X.conj().T
    return pref * G


def offset_average_eps2(inputs_list, weights, omega, eta):
    """k-offset averaged spectrum (§IV, k-point convergence): sum_o w_o eps2_o(omega), each
    eps2_o from an independent calculation on the dense mesh shifted by offset o (its own
    bands at the shifted k-points; Eq. abs_vel with its own prefactor)."""
    tot = np.zeros(len(omega))
    for inp, w in zip(inputs_list, weights):
        orc = BSEOracle(inp)
        tot += w * eps2_exact(orc.hamiltonian(), orc.dipoles(), omega, eta, orc.prefactor())
    return tot


def interp_V(V_R, R_W, w_RW, q):
    """V_mu,nu(q) = sum_R w_R Vbar_mu,nu(R) e^{-i q.R}: the bare interaction's companion of the
    W interpolation (the V kernel of §III.A with the dual-mesh R-sum of §III.B); at q = 0 it
    is the V(0) = sum_R Vbar(R) the exchange uses."""
    return interp_W(V_R, R_W, w_RW, q)

