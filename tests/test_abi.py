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


def test_noalloc_binding_rejects_bad_arguments_before_any_call():
    """ct_jacT_noalloc writes through raw pointers with the sizes it is given:
    the binding refuses wrong sizes, dtypes, element counts, strides and CPU
    tensors before calling it (dtype / count / stride checks come before the
    device check, so each is reached here with CPU tensors)."""
    torch = pytest.importorskip("torch")
    from paper_2605_06336_gb300 import ct
    N, B, V = 16, 23, 6
    f64, f32 = torch.float64, torch.float32
    good = dict(theta=torch.zeros(V, dtype=f64), delta=torch.zeros(V, dtype=f64), x=torch.zeros(N * N, dtype=f32),
                r=torch.zeros(V * B, dtype=f32), gtheta=torch.zeros(V, dtype=f64), gdelta=torch.zeros(V, dtype=f64))

    def call(N=N, B=B, V=V, **over):
        a = dict(good, **over)
        ct.ct_jacT_noalloc(N, B, V, a["theta"], a["delta"], a["x"], a["r"], a["gtheta"], a["gdelta"])

    for sizes in (dict(N=1), dict(B=0), dict(V=0), dict(N=ct.NOALLOC_MAX_N + 1), dict(B=ct.NOALLOC_MAX_BINS + 1),
                  dict(V=ct.NOALLOC_MAX_VIEWS + 1)):
        with pytest.raises(ValueError):
            call(**sizes)
    bad = {
        "theta": [None, torch.zeros(V, dtype=f32), torch.zeros(V + 1, dtype=f64), torch.zeros(2 * V, dtype=f64)[::2]],
        "delta": [torch.zeros(V, dtype=f32), torch.zeros(V - 1, dtype=f64)],
        "x": [None, torch.zeros(N * N, dtype=f64), torch.zeros(N * N, dtype=torch.float16), torch.zeros(N * N - 1, dtype=f32),
              torch.zeros(N, 2 * N, dtype=f32)[:, ::2]],
        "r": [None, torch.zeros(V * B, dtype=f64), torch.zeros(V * B + 1, dtype=f32)],
        "gtheta": [None, torch.zeros(V, dtype=f32), torch.zeros(V - 1, dtype=f64)],
        "gdelta": [torch.zeros(V, dtype=f32), torch.zeros(V + 1, dtype=f64)],
    }
    for name, values in bad.items():
        for v in values:
            with pytest.raises(ValueError, match=f"noalloc: {name} "):
                call(**{name: v})
    # everything well formed but on the host: refused as not CUDA
    with pytest.raises(ValueError, match="CUDA"):
        call()
    with pytest.raises(ValueError, match="CUDA"):
        call(delta=None, gdelta=None)
