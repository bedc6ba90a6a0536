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


def gpu_hamiltonian(inp, precision="fp64", alpha=2.0, Wq=False):
    import torch
    from paper_2607_05853_b300.api import BSE
    b = BSE.from_inputs(inp, precision=precision, alpha=alpha)
    d = to_dev(inp)
    Wq_out = torch.empty((b.nk, b.naux, b.naux), dtype=torch.complex128, device="cuda") if Wq else None
    b.interp_W(d["W_R"], d["V0"], Wq_out)
    b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
    H = b.assemble()
    b.sync()
    return b, d, H, Wq_out
