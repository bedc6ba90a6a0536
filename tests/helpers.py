"""Shared test helpers: move generator output to the device and run the library path."""
import numpy as np


def to_dev(inp):
    import torch
    d = {}
    for k in ("W_R", "V0", "C_R", "e_qp", "e_ks"):
        d[k] = torch.from_numpy(np.ascontiguousarray(inp[k], np.float64)).cuda()
    for k in ("c_k", "vel"):
        d[k] = torch.from_numpy(np.ascontiguousarray(inp[k], np.complex128)).cuda()
    return d


def gpu_hamiltonian(inp, precision="fp64", alpha=2.0, Wq=False, **kw):
    import torch
    from paper_2607_05853_b300.api import BSE
    b = BSE.from_inputs(inp, precision=precision, alpha=alpha, **kw)
    d = to_dev(inp)
    Wq_out = torch.empty((b.nk, b.naux, b.naux), dtype=torch.complex128, device="cuda") if Wq else None
    b.interp_W(d["W_R"], d["V0"], Wq_out)
    b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
    H = b.assemble()
    b.sync()
    return b, d, H, Wq_out


# ---- split-precision parity bounds ------------------------------------------------------------
# The diagonal of H (the 3-7 eV E_c - E_v plus its kernel terms) and the off-diagonal kernel
# terms (<~0.1 eV) are bounded separately, each relative to its own largest reference value:
# a bound relative to max|H| would be set by the diagonal and be ~50x too loose for the
# kernels.  Measured against the oracle (max error / max reference, over tiny, ragged, 2-D,
# Nv = Nc = 6, finite-Q and the 27648-dim sampled blocks):
#   off-diagonal  bf16x3 5.0e-7 .. 1.7e-6   bf16x2 3.8e-6 .. 1.1e-5   bf16x1 1.9e-3 .. 3.6e-3
#   diagonal      bf16x3 <= 4.7e-8          bf16x2 <= 2.6e-7          bf16x1 <= 9.0e-5
#   coupling B    bf16x3 4.9e-7 .. 6.1e-7   bf16x2 3.1e-6 .. 5.2e-6   bf16x1 1.4e-3 .. 2.7e-3
#   tf32x2        off-diagonal 4.0e-7 .. 7.4e-7, diagonal <= 4.7e-8, B 3.9e-7 .. 5.7e-7
# and on the 27648-dim sampled blocks: H bf16x3 1.7e-6 (bf16x2 3.8e-6, tf32x2 1.5e-6),
# H(Q) 2.3e-6, B 1.5e-6.  With N_aux = 185 (the unfused GEMM path) the off-diagonal errors are
# 1.1e-6 (bf16x3, tf32x2) and the diagonal ones 1.3e-7 .. 1.5e-7: there the diagonal's kernel
# terms, not its storage rounding, set its error, so the diagonal bound is the larger of the
# storage bound and the off-diagonal bound scaled to absolute (assert_split_close);
# the larger cell's blocks sum more ABFs, so the full-size bound is the wider SPLIT_OFF_FULL.
# The bf16x3 bounds sit between the bf16x3 and bf16x2 errors, so a build whose tensor-core
# GEMMs kept only bf16x2's three piece products fails them (tests/test_gpu_split.py checks
# that on the real bf16x2 path).  The diagonal bound is the complex64 storage rounding
# (2^-23 of the value) for bf16x3; the order-one kernel error of bf16x1 dominates its own.
# tf32x2 (two tf32 pieces, ~22 bits) carries the FP32 stages' error as bf16x3 does and takes its
# bounds; a tf32x2 GEMM that kept only the hi x hi product would be off by ~2^-11.
SPLIT_OFF = {"bf16x3": 3e-6, "bf16x2": 3e-5, "bf16x1": 1e-2, "tf32x2": 3e-6}
SPLIT_OFF_FULL = {"bf16x3": 3e-6, "tf32x2": 3e-6}   # the 27648-dim sampled blocks of H, H(Q) and B
SPLIT_DIAG = {"bf16x3": 1.2e-7, "bf16x2": 5e-7, "bf16x1": 1e-3, "tf32x2": 1.2e-7}
SPLIT_B = {"bf16x3": 1.5e-6, "bf16x2": 2e-5, "bf16x1": 1e-2, "tf32x2": 1.5e-6}


def offdiag_diag_errors(got, ref):
    """(max|got - ref| off the diagonal / max|ref| off the diagonal,
    max|got - ref| on the diagonal / max|ref| on the diagonal) of square matrices."""
    got = np.asarray(got, np.complex128)
    ref = np.asarray(ref, np.complex128)
    eye = np.eye(ref.shape[0], dtype=bool)
    d = np.abs(got - ref)
    off_scale = np.abs(ref[~eye]).max() if ref.shape[0] > 1 else 0.0
    off = d[~eye].max() / off_scale if off_scale > 0 else 0.0
    return off, d[eye].max() / np.abs(ref[eye]).max()


def assert_split_close(got, ref, prec, off_tol=None):
    """H parity of a split precision with the bounds above: the off-diagonal relative to its
    largest reference element; the diagonal within the larger of its storage bound (relative
    to the largest diagonal element) and the off-diagonal bound in absolute terms (the
    diagonal carries the same kernel terms)."""
    off, diag = offdiag_diag_errors(got, ref)
    ot = off_tol if off_tol is not None else SPLIT_OFF[prec]
    assert off <= ot, (prec, "off-diagonal", off)
    ref = np.asarray(ref, np.complex128)
    eye = np.eye(ref.shape[0], dtype=bool)
    dmax = np.abs(ref[eye]).max()
    omax = np.abs(ref[~eye]).max() if ref.shape[0] > 1 else 0.0
    assert diag * dmax <= max(SPLIT_DIAG[prec] * dmax, ot * omax), (prec, "diagonal", diag)
    return off, diag
