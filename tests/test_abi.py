"""The C ABI library loads and exports every symbol include/lss.h declares
(no GPU needed: no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lss.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(lss_\w+)\(", src, re.M)))


def _lib_path():
    from paper_1705_09443_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.LIB_PATH


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lss_setup", "lss_factor", "lss_solve", "lss_apply_A", "lss_apply_P",
                     "lss_plane_wave_rhs", "lss_destroy", "lss_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib_path())
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_1705_09443_gb300 import _lib
    assert sorted(_lib.SYMBOLS) == _declared()


def test_setup_argument_errors_without_gpu_work():
    """Argument validation happens before any device call."""
    from paper_1705_09443_gb300 import _lib
    lib = _lib.load()
    ctx = ctypes.c_void_p()
    p = _lib.Pml(4, 10.0)
    s = _lib.Slab(4, 0, 0)
    g = _lib.Grid(4, 16)
    rc = lib.lss_setup(ctypes.byref(ctx), ctypes.byref(g), 10.0, ctypes.c_void_p(16), ctypes.byref(p),
                       ctypes.byref(s), 0, None)
    assert rc == -1 and ctx.value is None and b"dim" in lib.lss_last_error(None)
    g = _lib.Grid(3, 200)          # 3D grids up to n = 128
    rc = lib.lss_setup(ctypes.byref(ctx), ctypes.byref(g), 10.0, ctypes.c_void_p(16), ctypes.byref(p),
                       ctypes.byref(s), 0, None)
    assert rc == -8 and ctx.value is None
    g = _lib.Grid(2, 16)
    rc = lib.lss_setup(ctypes.byref(ctx), ctypes.byref(g), -1.0, ctypes.c_void_p(16), ctypes.byref(p),
                       ctypes.byref(s), 0, None)
    assert rc == -1 and b"omega" in lib.lss_last_error(None)
    assert lib.lss_factor(None, None) == -1
    lib.lss_destroy(None)
