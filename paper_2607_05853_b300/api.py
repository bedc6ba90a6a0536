"""Thin Python binding of libbse (include/bse.h): argument checks and marshalling only.

Every step of the path runs in the CUDA library; torch supplies device memory and the
stream.  Method names follow the C entry points (bse_setup -> BSE(...),
bse_interp_W -> BSE.interp_W, ...).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

__all__ = ["BSE", "BseError", "launch_count", "batch_assemble", "batch_release"]

BseError = _lib.BseError


def launch_count() -> int:
    """Kernels launched by libbse in this process."""
    return int(_lib.load().bse_launch_count())


def _dev(t: torch.Tensor, dtype, name: str, numel: int | None = None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    return t.data_ptr()


class BSE:
    """One crystal's TDA-BSE problem bound to the current CUDA device and stream."""

    def __init__(self, *, nao, naux, dense, R_C, R_W, w_RW, nv, nc, k_offset=(0.0, 0.0, 0.0),
                 alpha=2.0, precision="fp64", h_complex128: bool = False, coarse=None, lattice=None,
                 stream: torch.cuda.Stream | None = None):
        lib = _lib.load()
        self._lib = lib
        nao = np.ascontiguousarray(nao, np.int32)
        naux = np.ascontiguousarray(naux, np.int32)
        R_C = np.ascontiguousarray(R_C, np.int32).reshape(-1, 3)
        R_W = np.ascontiguousarray(R_W, np.int32).reshape(-1, 3)
        w_RW = np.ascontiguousarray(w_RW, np.float64)
        if precision not in _lib.PRECISIONS:
            raise ValueError(f"precision must be one of {list(_lib.PRECISIONS)}")
        self.precision = precision
        p = _lib.BseParams()
        p.n_atoms = len(nao)
        p.nao_per_atom = nao.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        p.naux_per_atom = naux.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        p.dense[:] = [int(x) for x in dense]
        p.k_offset[:] = [float(x) for x in k_offset]
        p.n_RC = len(R_C)
        p.R_C = R_C.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        p.n_RW = len(R_W)
        p.R_W = R_W.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        p.w_RW = w_RW.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p.nv, p.nc = int(nv), int(nc)
        p.alpha = float(alpha)
        p.precision = _lib.PRECISIONS[precision]
        p.h_complex128 = 1 if h_complex128 else 0
        if coarse is not None:            # optional R-set checks (bse_params.coarse / lattice)
            p.coarse[:] = [int(x) for x in coarse]
        self._lattice = None if lattice is None else np.ascontiguousarray(lattice, np.float64).reshape(3, 3)
        if self._lattice is not None:
            p.lattice = self._lattice.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ctx = ctypes.c_void_p()
        st = lib.bse_setup(ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        if st != _lib.BSE_OK:
            raise BseError(st, "bse_setup rejected the parameters or could not allocate")
        self._ctx = ctx
        self.nk = int(np.prod(dense))
        self.nv, self.nc = int(nv), int(nc)
        self.nb = self.nv + self.nc
        self.dim = int(lib.bse_dim(ctx))
        self.naux = int(lib.bse_naux(ctx))
        self.nao = int(lib.bse_nao(ctx))
        self.n_RW = len(R_W)
        self.n_RC = len(R_C)
        self.h_dtype = torch.complex128 if (precision == "fp64" or h_complex128) else torch.complex64

    @classmethod
    def from_inputs(cls, inp: dict, **kw) -> "BSE":
        kw.setdefault("coarse", inp.get("coarse"))
        kw.setdefault("lattice", inp.get("lattice"))
        return cls(nao=inp["nao"], naux=inp["naux"], dense=inp["dense"], R_C=inp["R_C"], R_W=inp["R_W"],
                   w_RW=inp["w_RW"], nv=inp["nv"], nc=inp["nc"], k_offset=inp["k_offset"], **kw)

    # -- helpers -------------------------------------------------------------------------
    def _check(self, st: int, what: str):
        if st != _lib.BSE_OK:
            raise BseError(st, f"{what}: {self._lib.bse_last_error(self._ctx).decode()}")

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.bse_free(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the ABI -------------------------------------------------------------------------
    def interp_W(self, W_R: torch.Tensor, V0: torch.Tensor | None, Wq_out: torch.Tensor | None = None):
        """bse_interp_W.  V0 may be None once set_momentum has been given V_R."""
        na = self.naux
        a = _dev(W_R, torch.float64, "W_R", self.n_RW * na * na)
        b = _dev(V0, torch.float64, "V0", na * na) if V0 is not None else None
        c = _dev(Wq_out, torch.complex128, "Wq_out", self.nk * na * na) if Wq_out is not None else None
        self._check(self._lib.bse_interp_W(self._ctx, a, b, c), "bse_interp_W")
        return Wq_out

    def interp_V(self, V_R: torch.Tensor, Vq_out: torch.Tensor | None = None) -> torch.Tensor:
        """bse_interp_V: the bare interaction V(q) at every dense transfer q (complex128)."""
        if Vq_out is None:
            Vq_out = torch.empty((self.nk, self.naux, self.naux), dtype=torch.complex128, device="cuda")
        a = _dev(V_R, torch.float64, "V_R", self.n_RW * self.naux * self.naux)
        b = _dev(Vq_out, torch.complex128, "Vq_out", self.nk * self.naux * self.naux)
        self._check(self._lib.bse_interp_V(self._ctx, a, b), "bse_interp_V")
        return Vq_out

    def set_momentum(self, Q, V_R: torch.Tensor | None = None):
        """bse_set_momentum: exciton momentum Q (dense-mesh steps) and, for the exchange at
        Q != 0, the real-space bare interaction V_R."""
        q = (ctypes.c_int32 * 3)(*[int(x) for x in Q])
        v = None if V_R is None else _dev(V_R, torch.float64, "V_R", self.n_RW * self.naux * self.naux)
        self._check(self._lib.bse_set_momentum(self._ctx, ctypes.cast(q, ctypes.c_void_p), v),
                    "bse_set_momentum")

    def project_pairs(self, C_R: torch.Tensor, c_k: torch.Tensor, e_qp: torch.Tensor):
        a = _dev(C_R, torch.float64, "C_R", self.n_RC * self.nao * self.nao * self.naux)
        b = _dev(c_k, torch.complex128, "c_k", self.nk * self.nao * self.nb)
        c = _dev(e_qp, torch.float64, "e_qp", self.nk * self.nb)
        self._check(self._lib.bse_project_pairs(self._ctx, a, b, c), "bse_project_pairs")

    def assemble(self, H: torch.Tensor | None = None) -> torch.Tensor:
        if H is None:
            H = torch.empty((self.dim, self.dim), dtype=self.h_dtype, device="cuda")
        h = _dev(H, self.h_dtype, "H", self.dim * self.dim)
        self._check(self._lib.bse_assemble(self._ctx, h), "bse_assemble")
        return H

    def assemble_coupling(self, B: torch.Tensor | None = None) -> torch.Tensor:
        """bse_assemble_coupling: the full-BSE coupling block B (same layout and dtype as H)."""
        if B is None:
            B = torch.empty((self.dim, self.dim), dtype=self.h_dtype, device="cuda")
        b = _dev(B, self.h_dtype, "B", self.dim * self.dim)
        self._check(self._lib.bse_assemble_coupling(self._ctx, b), "bse_assemble_coupling")
        return B

    def dipole_vector(self, vel: torch.Tensor, e_ks: torch.Tensor, u: torch.Tensor | None = None) -> torch.Tensor:
        if u is None:
            u = torch.empty((3, self.dim), dtype=torch.complex128, device="cuda")
        a = _dev(vel, torch.complex128, "vel", 3 * self.dim)
        b = _dev(e_ks, torch.float64, "e_ks", self.nk * self.nb)
        c = _dev(u, torch.complex128, "u", 3 * self.dim)
        self._check(self._lib.bse_dipole_vector(self._ctx, a, b, c), "bse_dipole_vector")
        return u

    def spectrum(self, H: torch.Tensor, u: torch.Tensor, n_steps: int, omega: torch.Tensor, eta: float,
                 prefactor: float, eps2: torch.Tensor | None = None, ab: torch.Tensor | None = None):
        n_pol = u.shape[0] if u.dim() == 2 else 1
        if eps2 is None:
            eps2 = torch.empty(omega.numel(), dtype=torch.float64, device="cuda")
        h = _dev(H, self.h_dtype, "H", self.dim * self.dim)
        a = _dev(u, torch.complex128, "u", n_pol * self.dim)
        o = _dev(omega, torch.float64, "omega")
        e = _dev(eps2, torch.float64, "eps2", omega.numel())
        abp = _dev(ab, torch.float64, "ab", n_pol * 3 * n_steps) if ab is not None else None
        self._check(self._lib.bse_spectrum(self._ctx, h, a, n_pol, int(n_steps), o, omega.numel(), float(eta),
                                           float(prefactor), e, abp), "bse_spectrum")
        return eps2

    def spectrum_add(self, H: torch.Tensor, u: torch.Tensor, n_steps: int, omega: torch.Tensor, eta: float,
                     prefactor: float, weight: float, eps2_acc: torch.Tensor):
        """bse_spectrum_add: eps2_acc += weight * spectrum (eps2_acc is read and written)."""
        n_pol = u.shape[0] if u.dim() == 2 else 1
        h = _dev(H, self.h_dtype, "H", self.dim * self.dim)
        a = _dev(u, torch.complex128, "u", n_pol * self.dim)
        o = _dev(omega, torch.float64, "omega")
        e = _dev(eps2_acc, torch.float64, "eps2_acc", omega.numel())
        self._check(self._lib.bse_spectrum_add(self._ctx, h, a, n_pol, int(n_steps), o, omega.numel(), float(eta),
                                               float(prefactor), float(weight), e), "bse_spectrum_add")
        return eps2_acc

    def spectrum_static(self, H: torch.Tensor, u: torch.Tensor, n_steps: int, omega: torch.Tensor, eta: float,
                        prefactor: float, eps2: torch.Tensor, ab: torch.Tensor | None = None):
        """bse_spectrum_static: the spectrum without any device allocation (outputs supplied)."""
        n_pol = u.shape[0] if u.dim() == 2 else 1
        h = _dev(H, self.h_dtype, "H", self.dim * self.dim)
        a = _dev(u, torch.complex128, "u", n_pol * self.dim)
        o = _dev(omega, torch.float64, "omega")
        e = _dev(eps2, torch.float64, "eps2", omega.numel())
        abp = _dev(ab, torch.float64, "ab", n_pol * 3 * n_steps) if ab is not None else None
        self._check(self._lib.bse_spectrum_static(self._ctx, h, a, n_pol, int(n_steps), o, omega.numel(), float(eta),
                                                  float(prefactor), e, abp), "bse_spectrum_static")
        return eps2

    def lowest(self, H: torch.Tensor, n_eig: int, n_steps: int, seed: int = 12345, vectors: bool = False):
        om = torch.empty(n_eig, dtype=torch.float64, device="cuda")
        rs = torch.empty(n_eig, dtype=torch.float64, device="cuda")
        vec = torch.empty((n_eig, self.dim), dtype=torch.complex128, device="cuda") if vectors else None
        h = _dev(H, self.h_dtype, "H", self.dim * self.dim)
        self._check(self._lib.bse_lowest(self._ctx, h, int(n_eig), int(n_steps), ctypes.c_uint64(seed),
                                         om.data_ptr(), rs.data_ptr(), vec.data_ptr() if vectors else None),
                    "bse_lowest")
        return (om, rs, vec) if vectors else (om, rs)

    def spectrum_matfree(self, u: torch.Tensor, n_steps: int, omega: torch.Tensor, eta: float, prefactor: float,
                         eps2: torch.Tensor | None = None, ab: torch.Tensor | None = None) -> torch.Tensor:
        """bse_spectrum_matfree: the Haydock spectrum with H recomputed per Lanczos product."""
        n_pol = u.shape[0] if u.dim() == 2 else 1
        if eps2 is None:
            eps2 = torch.empty(omega.numel(), dtype=torch.float64, device="cuda")
        uu = _dev(u, torch.complex128, "u", n_pol * self.dim)
        om = _dev(omega, torch.float64, "omega")
        e = _dev(eps2, torch.float64, "eps2", omega.numel())
        a = _dev(ab, torch.float64, "ab", n_pol * 3 * n_steps) if ab is not None else None
        self._check(self._lib.bse_spectrum_matfree(self._ctx, uu, int(n_pol), int(n_steps), om, int(omega.numel()),
                                                   float(eta), float(prefactor), e, a), "bse_spectrum_matfree")
        return eps2

    def spectrum_full(self, A: torch.Tensor, B: torch.Tensor, u: torch.Tensor, n_steps: int, omega: torch.Tensor,
                      eta: float, prefactor: float, eps2: torch.Tensor | None = None) -> torch.Tensor:
        """bse_spectrum_full: eps2 of the full BSE (X and Y amplitudes)."""
        n_pol = u.shape[0] if u.dim() == 2 else 1
        if eps2 is None:
            eps2 = torch.empty(omega.numel(), dtype=torch.float64, device="cuda")
        a = _dev(A, self.h_dtype, "A", self.dim * self.dim)
        b = _dev(B, self.h_dtype, "B", self.dim * self.dim)
        uu = _dev(u, torch.complex128, "u", n_pol * self.dim)
        om = _dev(omega, torch.float64, "omega")
        e = _dev(eps2, torch.float64, "eps2", omega.numel())
        self._check(self._lib.bse_spectrum_full(self._ctx, a, b, uu, int(n_pol), int(n_steps), om, int(omega.numel()),
                                                float(eta), float(prefactor), e), "bse_spectrum_full")
        return eps2

    def lowest_full(self, A: torch.Tensor, B: torch.Tensor, n_eig: int, n_steps: int, seed: int = 12345):
        """bse_lowest_full: the lowest positive full-BSE excitation energies and residual bounds."""
        om = torch.empty(n_eig, dtype=torch.float64, device="cuda")
        rs = torch.empty(n_eig, dtype=torch.float64, device="cuda")
        a = _dev(A, self.h_dtype, "A", self.dim * self.dim)
        b = _dev(B, self.h_dtype, "B", self.dim * self.dim)
        self._check(self._lib.bse_lowest_full(self._ctx, a, b, int(n_eig), int(n_steps), ctypes.c_uint64(seed),
                                              om.data_ptr(), rs.data_ptr()), "bse_lowest_full")
        return om, rs

    def adjoint_seed(self, vecs: torch.Tensor, g: torch.Tensor, Gamma: torch.Tensor | None = None):
        r = vecs.shape[0]
        if Gamma is None:
            Gamma = torch.empty((self.dim, self.dim), dtype=torch.complex128, device="cuda")
        a = _dev(vecs, torch.complex128, "vecs", r * self.dim)
        b = _dev(g, torch.float64, "g", r)
        c = _dev(Gamma, torch.complex128, "Gamma", self.dim * self.dim)
        self._check(self._lib.bse_adjoint_seed(self._ctx, a, b, int(r), c), "bse_adjoint_seed")
        return Gamma

    def window_seed(self, H: torch.Tensor, u: torch.Tensor, n_steps: int, w_lo: float, w_hi: float, eta: float,
                    prefactor: float, Gamma: torch.Tensor | None = None):
        """bse_window_seed: (Gamma, I) for I = the spectrum integrated over [w_lo, w_hi]."""
        n_pol = u.shape[0] if u.dim() == 2 else 1
        if Gamma is None:
            Gamma = torch.empty((self.dim, self.dim), dtype=torch.complex128, device="cuda")
        I = torch.empty(1, dtype=torch.float64, device="cuda")
        h = _dev(H, self.h_dtype, "H", self.dim * self.dim)
        a = _dev(u, torch.complex128, "u", n_pol * self.dim)
        c = _dev(Gamma, torch.complex128, "Gamma", self.dim * self.dim)
        self._check(self._lib.bse_window_seed(self._ctx, h, a, n_pol, int(n_steps), float(w_lo), float(w_hi),
                                              float(eta), float(prefactor), I.data_ptr(), c), "bse_window_seed")
        return Gamma, I

    def adjoint(self, Gamma: torch.Tensor, dW_R: torch.Tensor | None = None, de_qp: torch.Tensor | None = None):
        if dW_R is None:
            dW_R = torch.empty((self.n_RW, self.naux, self.naux), dtype=torch.float64, device="cuda")
        if de_qp is None:
            de_qp = torch.empty((self.nk, self.nb), dtype=torch.float64, device="cuda")
        a = _dev(Gamma, torch.complex128, "Gamma", self.dim * self.dim)
        b = _dev(dW_R, torch.float64, "dW_R", self.n_RW * self.naux * self.naux)
        c = _dev(de_qp, torch.float64, "de_qp", self.nk * self.nb)
        self._check(self._lib.bse_adjoint(self._ctx, a, b, c), "bse_adjoint")
        return dW_R, de_qp

    def profile(self, enable: bool = True):
        self._check(self._lib.bse_profile(self._ctx, int(enable)), "bse_profile")

    def profile_read(self, kernel: str):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self._lib.bse_profile_read(self._ctx, _lib.KERNEL_IDS[kernel], ctypes.byref(ms), ctypes.byref(n)),
                    "bse_profile_read")
        return ms.value, n.value

    def autotune(self, with_projection: bool = False):
        """bse_autotune: the chosen GEMM N tile (and, if asked, the projection's threads per block)."""
        chosen, proj = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.bse_autotune(self._ctx, ctypes.byref(chosen), ctypes.byref(proj)), "bse_autotune")
        return (chosen.value, proj.value) if with_projection else chosen.value

    def sync(self, timeout_ms: int = 600_000):
        """bse_sync: wait (at most timeout_ms; negative = no limit) and read the error word."""
        self._check(self._lib.bse_sync(self._ctx, int(timeout_ms)), "bse_sync")

    def selftest_delay(self, ms: int):
        """bse_selftest_delay: keep the stream busy for ms milliseconds (a host function)."""
        self._check(self._lib.bse_selftest_delay(self._ctx, int(ms)), "bse_selftest_delay")

    def selftest_wait(self, cycles: int):
        """bse_selftest_wait: one bounded device wait on a barrier nothing completes."""
        self._check(self._lib.bse_selftest_wait(self._ctx, int(cycles)), "bse_selftest_wait")


def batch_assemble(systems, Hs, stream=None, stamps: bool = False, schedule: str = "worklist"):
    """bse_batch_assemble: assemble several crystals as one CUDA graph.

    systems: list of BSE contexts (each past project_pairs); Hs: matching H tensors;
    schedule: "worklist" (grouped tensor-core launches over the systems' tiles, one split
    precision for all) or "chains" (each system's assembly on one of two concurrent chains).
    Returns per-system completion times in ns from the replay start when stamps=True."""
    lib = _lib.load()
    n = len(systems)
    for b, H in zip(systems, Hs):
        _dev(H, b.h_dtype, "H", b.dim * b.dim)
    ctxs = (ctypes.c_void_p * n)(*[b._ctx.value for b in systems])
    hp = (ctypes.c_void_p * n)(*[H.data_ptr() for H in Hs])
    st = stream if stream is not None else torch.cuda.current_stream()
    out = (ctypes.c_int64 * n)() if stamps else None
    if schedule not in _lib.BATCH_SCHEDULES:
        raise ValueError(f"schedule must be one of {list(_lib.BATCH_SCHEDULES)}")
    r = lib.bse_batch_assemble(ctxs, hp, n, ctypes.c_void_p(st.cuda_stream), _lib.BATCH_SCHEDULES[schedule], out)
    if r != _lib.BSE_OK:
        raise BseError(r, "bse_batch_assemble: " + lib.bse_last_error(systems[0]._ctx).decode())
    return [int(x) for x in out] if stamps else None


def batch_release():
    _lib.load().bse_batch_release()
