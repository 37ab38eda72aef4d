"""The C-ABI library loads and exports every symbol include/ctgb.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?(?:int|void|const char\s*\*)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ct_init", "ct_forward", "ct_adjoint", "ct_forward_repeat", "ct_adjoint_repeat", "ct_jac",
                     "ct_jacT", "ct_destroy", "ct_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2605_06336_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.ct_strerror.restype = ctypes.c_char_p
    assert lib.ct_strerror(0) == b"ok"
    assert b"argument" in lib.ct_strerror(-1)


def test_init_rejects_bad_geometry_without_touching_the_gpu():
    from paper_2605_06336_gb300 import ct
    lib = ct.load_library()
    g = ct.ct_geom()
    g.N, g.B, g.n_views, g.n_frames, g.max_batch, g.precision = 0, 3, 1, 1, 1, 0
    h = ctypes.c_void_p()
    assert lib.ct_init(ctypes.byref(g), None, ctypes.byref(h)) == ct.CT_ERR_ARG
    g.N, g.precision = 16, 7
    assert lib.ct_init(ctypes.byref(g), None, ctypes.byref(h)) == ct.CT_ERR_ARG
    g.precision = 0
    for D in (-1.0, 5.0, float("inf"), float("nan")):  # fan source inside the image disc, or not finite
        g.source_distance = D
        assert lib.ct_init(ctypes.byref(g), None, ctypes.byref(h)) == ct.CT_ERR_ARG
    assert lib.ct_forward(None, None, None, None, None, 1) == ct.CT_ERR_ARG
