"""The C ABI library on a machine without a GPU: it loads, exports every symbol that
include/bse.h declares, and rejects bad parameters before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_05853_b300 import build, _lib
    build.build()
    return _lib.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "bse.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bse_[a-zA-Z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 14
    for s in syms:
        assert hasattr(lib, s), s
    from paper_2607_05853_b300 import _lib
    assert sorted(_lib.EXPORTS) == syms


def _params(**over):
    from paper_2607_05853_b300 import _lib
    keep = {}
    nao = np.array([4, 4], np.int32)
    naux = np.array([20, 20], np.int32)
    RC = np.zeros((1, 3), np.int32)
    RW = np.zeros((1, 3), np.int32)
    w = np.ones(1)
    keep.update(nao=nao, naux=naux, RC=RC, RW=RW, w=w)
    p = _lib.BseParams()
    p.n_atoms = 2
    p.nao_per_atom = nao.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p.naux_per_atom = naux.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p.dense[:] = [4, 4, 4]
    p.k_offset[:] = [0.0, 0.0, 0.0]
    p.n_RC, p.R_C = 1, RC.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p.n_RW, p.R_W = 1, RW.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p.w_RW = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.nv, p.nc, p.alpha, p.precision = 4, 4, 2.0, 0
    for k, v in over.items():
        setattr(p, k, v)
    return p, keep


@pytest.mark.parametrize("field,value", [("nv", 0), ("nc", 9), ("nv", 5), ("n_atoms", 0), ("precision", 7),
                                         ("n_RC", 0), ("n_RW", 0), ("alpha", float("nan"))])
def test_bad_parameters_rejected_without_device(lib, field, value):
    from paper_2607_05853_b300 import _lib
    p, keep = _params(**{field: value})
    if field == "nv" and value == 5:
        p.nc = 4  # nv + nc = 9 > 8 NAOs
    ctx = ctypes.c_void_p(123)
    st = lib.bse_setup(ctypes.byref(p), None, ctypes.byref(ctx))
    assert st == _lib.BSE_EINVAL
    assert ctx.value is None


def test_bad_mesh_rejected(lib):
    from paper_2607_05853_b300 import _lib
    p, keep = _params()
    p.dense[:] = [4, 0, 4]
    ctx = ctypes.c_void_p()
    assert lib.bse_setup(ctypes.byref(p), None, ctypes.byref(ctx)) == _lib.BSE_EINVAL
    assert lib.bse_setup(None, None, ctypes.byref(ctx)) == _lib.BSE_EINVAL


def test_null_context_calls_are_safe(lib):
    from paper_2607_05853_b300 import _lib
    lib.bse_free(None)
    assert lib.bse_last_error(None) == b"null context"
    assert lib.bse_dim(None) == -1
    assert lib.bse_sync(None, 0) == _lib.BSE_EINVAL
    assert lib.bse_selftest_delay(None, 1) == _lib.BSE_EINVAL
    assert lib.bse_selftest_wait(None, 1) == _lib.BSE_EINVAL
    assert lib.bse_assemble(None, None) == _lib.BSE_EINVAL
    assert lib.bse_launch_count() >= 0


def test_extension_entries_reject_null_context(lib):
    """The full-BSE, finite-momentum, matrix-free and V(q) entries refuse a null context
    before touching the device."""
    from paper_2607_05853_b300 import _lib
    q = (ctypes.c_int32 * 3)(1, 0, 0)
    assert lib.bse_set_momentum(None, ctypes.cast(q, ctypes.c_void_p), None) == _lib.BSE_EINVAL
    assert lib.bse_assemble_coupling(None, None) == _lib.BSE_EINVAL
    assert lib.bse_spectrum_full(None, None, None, None, 1, 2, None, 1, 0.1, 1.0, None) == _lib.BSE_EINVAL
    assert lib.bse_lowest_full(None, None, None, 1, 2, 1, None, None) == _lib.BSE_EINVAL
    assert lib.bse_spectrum_matfree(None, None, 1, 2, None, 1, 0.1, 1.0, None, None) == _lib.BSE_EINVAL
    assert lib.bse_interp_V(None, None, None) == _lib.BSE_EINVAL


def _params_from(inp, coarse=True, lattice=True):
    from paper_2607_05853_b300 import _lib
    keep = {k: np.ascontiguousarray(inp[k], dt) for k, dt in
            (("nao", np.int32), ("naux", np.int32), ("R_C", np.int32), ("R_W", np.int32), ("w_RW", np.float64),
             ("lattice", np.float64))}
    p = _lib.BseParams()
    p.n_atoms = len(keep["nao"])
    p.nao_per_atom = keep["nao"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p.naux_per_atom = keep["naux"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p.dense[:] = [int(x) for x in inp["dense"]]
    p.k_offset[:] = [float(x) for x in inp["k_offset"]]
    p.n_RC, p.R_C = len(keep["R_C"]), keep["R_C"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p.n_RW, p.R_W = len(keep["R_W"]), keep["R_W"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p.w_RW = keep["w_RW"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.nv, p.nc, p.alpha, p.precision = int(inp["nv"]), int(inp["nc"]), 2.0, 1
    if coarse:
        p.coarse[:] = [int(x) for x in inp["coarse"]]
    if lattice:
        p.lattice = keep["lattice"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return p, keep


def _inputs(which):
    from synth import config_spec, make_inputs, batched_specs
    from synth.crystal import CrystalSpec, _hex
    if which == "tiny":
        return make_inputs(config_spec(0))
    if which == "batch":
        return make_inputs(batched_specs(16)[3])
    return make_inputs(CrystalSpec("2d", _hex(3.19, 20.0), np.array([[0, 0, 0], [1 / 3, 2 / 3, 0.08]]),
                                   (3, 4), (7, 6), (3, 3, 1), (6, 6, 1), 2, 2, 1717, two_d=True))


@pytest.mark.parametrize("which", ["tiny", "batch", "two_d"])
def test_coarse_mesh_and_lattice_checks(lib, which):
    """The R-set of W is the Wigner-Seitz folding of the coarse mesh (§III.B): the generator's
    sets pass bse_check_params with the coarse mesh and lattice given; a weight changed, a
    class left out or an image moved to a longer member of its class are rejected."""
    from paper_2607_05853_b300 import _lib
    inp = _inputs(which)
    p, keep = _params_from(inp)
    assert lib.bse_check_params(ctypes.byref(p)) == _lib.BSE_OK
    # a weight off by 10 %
    keep["w_RW"][0] *= 0.9
    assert lib.bse_check_params(ctypes.byref(p)) == _lib.BSE_EINVAL
    keep["w_RW"][0] /= 0.9
    # one class missing
    p.n_RW = len(keep["R_W"]) - 1
    assert lib.bse_check_params(ctypes.byref(p)) == _lib.BSE_EINVAL
    p.n_RW = len(keep["R_W"])
    # the longest image moved by one coarse period along a periodic axis: weights still sum to
    # one per class (it stays in its class), but it is no longer a shortest member
    lat = keep["lattice"]
    lens = np.linalg.norm(keep["R_W"] @ lat, axis=1)
    i = int(np.argmax(lens))
    ax = 0
    step = np.zeros(3, np.int32)
    step[ax] = int(inp["coarse"][ax]) * (1 if (keep["R_W"][i] @ lat) @ lat[ax] >= 0 else -1)
    keep["R_W"][i] += step
    assert lib.bse_check_params(ctypes.byref(p)) == _lib.BSE_EINVAL
    p.lattice = None                       # without the lattice only the weights are checked
    assert lib.bse_check_params(ctypes.byref(p)) == _lib.BSE_OK
    keep["R_W"][i] -= step
    p.coarse[:] = [int(inp["coarse"][0]) + 1, int(inp["coarse"][1]), int(inp["coarse"][2])]
    assert lib.bse_check_params(ctypes.byref(p)) == _lib.BSE_EINVAL   # the wrong coarse mesh
    p.coarse[:] = [0, 0, 0]
    assert lib.bse_check_params(ctypes.byref(p)) == _lib.BSE_OK       # not given: not checked
