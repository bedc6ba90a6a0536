"""ctypes declarations of the C ABI in include/bse.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_uint64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbse.so")

BSE_OK, BSE_EINVAL, BSE_ENOMEM, BSE_ECUDA, BSE_ETIMEOUT, BSE_ESTATE, BSE_EDEVICE = range(7)
STATUS_NAMES = ["BSE_OK", "BSE_EINVAL", "BSE_ENOMEM", "BSE_ECUDA", "BSE_ETIMEOUT", "BSE_ESTATE", "BSE_EDEVICE"]
PRECISIONS = {"fp64": 0, "bf16x3": 1, "bf16x2": 2, "bf16x1": 3, "tf32x2": 4}

# Every symbol include/bse.h declares.
EXPORTS = ["bse_check_params", "bse_setup", "bse_interp_W", "bse_project_pairs", "bse_assemble", "bse_dipole_vector",
           "bse_spectrum", "bse_lowest", "bse_sync", "bse_last_error", "bse_dim", "bse_naux",
           "bse_nao", "bse_launch_count", "bse_free", "bse_profile", "bse_profile_read",
           "bse_spectrum_static", "bse_adjoint_seed", "bse_adjoint", "bse_batch_assemble",
           "bse_batch_release", "bse_autotune", "bse_window_seed", "bse_spectrum_add", "bse_interp_V",
           "bse_set_momentum", "bse_assemble_coupling", "bse_spectrum_full", "bse_lowest_full",
           "bse_spectrum_matfree", "bse_selftest_delay", "bse_selftest_wait"]
BATCH_SCHEDULES = {"worklist": 0, "chains": 1}
KERNEL_IDS = {"interp": 0, "half": 1, "project": 2, "g1": 3, "g2": 4, "exch": 5, "matvec": 6, "reorth": 7}


class BseParams(ctypes.Structure):
    _fields_ = [
        ("n_atoms", c_int32),
        ("nao_per_atom", POINTER(c_int32)),
        ("naux_per_atom", POINTER(c_int32)),
        ("dense", c_int32 * 3),
        ("k_offset", c_double * 3),
        ("n_RC", c_int32),
        ("R_C", POINTER(c_int32)),
        ("n_RW", c_int32),
        ("R_W", POINTER(c_int32)),
        ("w_RW", POINTER(c_double)),
        ("nv", c_int32),
        ("nc", c_int32),
        ("alpha", c_double),
        ("precision", c_int32),
        ("h_complex128", c_int32),
        ("coarse", c_int32 * 3),
        ("lattice", POINTER(c_double)),
    ]


class BseError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


_lib = None


def load() -> ctypes.CDLL:
    """Load libbse.so from the package directory; fail loudly if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libbse.so not built ({LIB_PATH}); run paper_2607_05853_b300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp = c_void_p
    lib.bse_setup.argtypes = [POINTER(BseParams), vp, POINTER(vp)]
    lib.bse_check_params.argtypes = [POINTER(BseParams)]
    lib.bse_check_params.restype = c_int
    lib.bse_interp_W.argtypes = [vp, vp, vp, vp]
    lib.bse_interp_V.argtypes = [vp, vp, vp]
    lib.bse_set_momentum.argtypes = [vp, vp, vp]
    lib.bse_assemble_coupling.argtypes = [vp, vp]
    lib.bse_spectrum_full.argtypes = [vp, vp, vp, vp, c_int, c_int, vp, c_int, c_double, c_double, vp]
    lib.bse_lowest_full.argtypes = [vp, vp, vp, c_int, c_int, c_uint64, vp, vp]
    lib.bse_spectrum_matfree.argtypes = [vp, vp, c_int, c_int, vp, c_int, c_double, c_double, vp, vp]
    lib.bse_project_pairs.argtypes = [vp, vp, vp, vp]
    lib.bse_assemble.argtypes = [vp, vp]
    lib.bse_dipole_vector.argtypes = [vp, vp, vp, vp]
    lib.bse_spectrum.argtypes = [vp, vp, vp, c_int, c_int, vp, c_int, c_double, c_double, vp, vp]
    lib.bse_spectrum_static.argtypes = [vp, vp, vp, c_int, c_int, vp, c_int, c_double, c_double, vp, vp]
    lib.bse_spectrum_add.argtypes = [vp, vp, vp, c_int, c_int, vp, c_int, c_double, c_double, c_double, vp]
    lib.bse_lowest.argtypes = [vp, vp, c_int, c_int, c_uint64, vp, vp, vp]
    lib.bse_adjoint_seed.argtypes = [vp, vp, vp, c_int, vp]
    lib.bse_adjoint.argtypes = [vp, vp, vp, vp]
    lib.bse_window_seed.argtypes = [vp, vp, vp, c_int, c_int, c_double, c_double, c_double, c_double, vp, vp]
    lib.bse_batch_assemble.argtypes = [POINTER(vp), POINTER(vp), c_int, vp, c_int32, POINTER(c_int64)]
    lib.bse_batch_assemble.restype = c_int
    lib.bse_batch_release.argtypes = []
    lib.bse_batch_release.restype = None
    lib.bse_autotune.argtypes = [vp, POINTER(c_int), POINTER(c_int)]
    lib.bse_autotune.restype = c_int
    lib.bse_sync.argtypes = [vp, c_int32]
    lib.bse_selftest_delay.argtypes = [vp, c_int32]
    lib.bse_selftest_delay.restype = c_int
    lib.bse_selftest_wait.argtypes = [vp, c_int64]
    lib.bse_selftest_wait.restype = c_int
    lib.bse_last_error.argtypes = [vp]
    lib.bse_last_error.restype = ctypes.c_char_p
    lib.bse_dim.argtypes = [vp]
    lib.bse_dim.restype = c_int64
    lib.bse_naux.argtypes = [vp]
    lib.bse_naux.restype = c_int32
    lib.bse_nao.argtypes = [vp]
    lib.bse_nao.restype = c_int32
    lib.bse_launch_count.argtypes = []
    lib.bse_launch_count.restype = c_int64
    lib.bse_free.argtypes = [vp]
    lib.bse_free.restype = None
    lib.bse_profile.argtypes = [vp, c_int]
    lib.bse_profile.restype = c_int
    lib.bse_profile_read.argtypes = [vp, c_int, POINTER(c_double), POINTER(c_int64)]
    lib.bse_profile_read.restype = c_int
    for name in ("bse_setup", "bse_interp_W", "bse_project_pairs", "bse_assemble", "bse_dipole_vector",
                 "bse_spectrum", "bse_spectrum_static", "bse_lowest", "bse_adjoint_seed", "bse_adjoint",
                 "bse_window_seed", "bse_spectrum_add", "bse_interp_V", "bse_sync"):
        getattr(lib, name).restype = c_int
    _lib = lib
    return lib
