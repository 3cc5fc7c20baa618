"""ctypes binding of liblss.so (the C ABI declared in include/lss.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblss.so")

LSS_FP64, LSS_MIXED = 0, 1
ERRORS = {
    0: "LSS_OK", -1: "LSS_ERR_ARG", -2: "LSS_ERR_OOM", -3: "LSS_ERR_STATE", -4: "LSS_ERR_SINGULAR",
    -5: "LSS_ERR_NOCONVERGE", -6: "LSS_ERR_TIMEOUT", -7: "LSS_ERR_CUDA", -8: "LSS_ERR_UNSUPPORTED",
}

# every symbol include/lss.h declares
SYMBOLS = [
    "lss_setup", "lss_set_medium", "lss_factor", "lss_plane_wave_rhs", "lss_apply_A", "lss_apply_P", "lss_solve",
    "lss_adjoint_solve", "lss_medium_gradient", "lss_helmholtz_solve", "lss_solve_host", "lss_apply_slab", "lss_apply_slab_noalloc", "lss_info", "lss_slab_info", "lss_get_stencils",
    "lss_profile", "lss_profile_read", "lss_set_graphs", "lss_graph_count", "lss_autotune", "lss_setup_batch", "lss_batch_info", "lss_batch_instance", "lss_test_inject", "lss_last_error",
    "lss_destroy",
]
PROF_CATEGORIES = ["matvec", "sparsify", "slab_a", "recur", "slab_e", "factor", "iface", "krylov", "setup"]


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int)]


class Pml(ctypes.Structure):
    _fields_ = [("b_pml", ctypes.c_int), ("C", ctypes.c_double)]


class Slab(ctypes.Structure):
    _fields_ = [("b_slab", ctypes.c_int), ("b_aux", ctypes.c_int), ("n_samples", ctypes.c_int), ("fronts", ctypes.c_int),
                ("recursive", ctypes.c_int)]


class Gmres(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("relres_est", ctypes.c_double),
                ("relres_true", ctypes.c_double)]


class LssError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load() -> ctypes.CDLL:
    """Load liblss.so (built by build.py / __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1705_09443_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    lib.lss_setup.argtypes = [P(vp), P(Grid), d, vp, P(Pml), P(Slab), i, vp]
    lib.lss_set_medium.argtypes = [vp, vp, vp]
    lib.lss_factor.argtypes = [vp, vp]
    lib.lss_profile.argtypes = [vp, i]
    lib.lss_profile_read.argtypes = [vp, vp, vp, i]
    lib.lss_set_graphs.argtypes = [vp, i]
    lib.lss_graph_count.argtypes = [vp, P(i), P(i)]
    lib.lss_autotune.argtypes = [vp, i, P(i), vp]
    lib.lss_plane_wave_rhs.argtypes = [vp, vp, i, vp, vp, vp]
    lib.lss_apply_A.argtypes = [vp, vp, vp, i, i, vp]
    lib.lss_apply_P.argtypes = [vp, vp, vp, i, i, vp]
    lib.lss_solve.argtypes = [vp, vp, vp, i, P(Gmres), P(Stats), vp]
    lib.lss_solve_host.argtypes = [vp, vp, vp, i, P(Gmres), P(Stats), vp]
    lib.lss_adjoint_solve.argtypes = [vp, vp, vp, i, P(Gmres), P(Stats), vp]
    lib.lss_medium_gradient.argtypes = [vp, vp, vp, vp, i, vp, vp]
    lib.lss_helmholtz_solve.argtypes = [vp, vp, vp, i, P(Gmres), P(Stats), vp]
    lib.lss_apply_slab.argtypes = [vp, i, vp, vp, i, vp]
    lib.lss_apply_slab_noalloc.argtypes = [vp, i, vp, vp, i, vp]
    lib.lss_info.argtypes = [vp, P(i), P(i), P(i)]
    lib.lss_slab_info.argtypes = [vp, i, P(i), P(i), P(i)]
    lib.lss_get_stencils.argtypes = [vp, vp, vp]
    lib.lss_setup_batch.argtypes = [P(vp), i, P(Grid), P(d), P(vp), P(Pml), P(Slab), i, vp]
    lib.lss_batch_info.argtypes = [vp, P(i), P(ctypes.c_longlong)]
    lib.lss_batch_instance.argtypes = [vp, i, P(vp)]
    lib.lss_test_inject.argtypes = [vp, i, i, ctypes.c_longlong, vp]
    lib.lss_last_error.argtypes = [vp]
    lib.lss_last_error.restype = ctypes.c_char_p
    lib.lss_destroy.argtypes = [vp]
    lib.lss_destroy.restype = None
    for name in SYMBOLS:
        if name not in ("lss_last_error", "lss_destroy"):
            getattr(lib, name).restype = i
    _lib = lib
    return lib


def check(code: int, ctx=None) -> int:
    if code in (0,):
        return code
    lib = load()
    msg = lib.lss_last_error(ctx)
    raise LssError(code, msg.decode() if msg else "")
