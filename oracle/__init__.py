"""FP64 CPU oracle for the angle-dependent CT operator and the NL-RMM-GKS solver.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path of ``paper_2605_06336_gb300`` and never imports it.

``ct_oracle.c`` holds the operator arithmetic (Joseph line integrals, a
scatter-form transpose, the analytic angle/offset derivatives, for the
parallel beam and the fan beam); this module
compiles it with gcc and wraps it with numpy.  ``nlrmm.py`` holds the solver
(MM-GKS / RMM-GKS / NL-RMM-GKS, Sec. 3-4 and the supplementary algorithms).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ct_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_ct.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ct_oracle.c into a shared library next to it (plain -O2, no -ffast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        lib.orc_forward.argtypes = [I, I, I, P, P, P, P, P]
        lib.orc_adjoint.argtypes = [I, I, I, I, P, P, P, P, P]
        lib.orc_dsample.argtypes = [I, I, I, P, P, P, P, P, P]
        lib.orc_jac.argtypes = [I, I, I, P, P, P, P, P, P, P]
        lib.orc_jacT.argtypes = [I, I, I, P, P, P, P, P, P, P]
        D = ctypes.c_double
        lib.orc_fan_forward.argtypes = [I, I, I, P, D, P, P, P, P]
        lib.orc_fan_adjoint.argtypes = [I, I, I, I, P, D, P, P, P, P]
        lib.orc_fan_dsample.argtypes = [I, I, I, P, D, P, P, P, P, P]
        for f in (lib.orc_forward, lib.orc_adjoint, lib.orc_dsample, lib.orc_jac, lib.orc_jacT,
                  lib.orc_fan_forward, lib.orc_fan_adjoint, lib.orc_fan_dsample):
            f.restype = None
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Geometry:
    """Geometry: N x N image, B bins, per-view frame index.

    ``views_per_frame`` splits the flat view list into consecutive frames
    (block-diagonal operator of the dynamic problem); ``None`` = one frame.
    ``fan_D``: parallel beam when None, else fan beam with the source at
    distance fan_D (pixels) from the rotation centre (``ct_oracle.c``).
    """

    def __init__(self, N: int, B: int, n_views: int, views_per_frame=None, fan_D=None):
        self.N, self.B, self.V = int(N), int(B), int(n_views)
        self.fan_D = None if fan_D is None else float(fan_D)
        if views_per_frame is None:
            self.F = 1
            self.fov = None
        else:
            vpf = [int(x) for x in views_per_frame]
            if sum(vpf) != self.V:
                raise ValueError("views_per_frame must sum to n_views")
            self.F = len(vpf)
            self.fov = np.ascontiguousarray(np.repeat(np.arange(self.F), vpf), dtype=np.int32)

    @property
    def n(self):
        return self.F * self.N * self.N

    @property
    def m(self):
        return self.V * self.B


def forward(g: Geometry, theta, X, delta=None):
    """Y = H(theta, delta) X.  X: (F*N*N,) or (K, F*N*N) -> Y: (V*B,) or (K, V*B)."""
    lib = _load()
    X = _f64(X)
    th = _f64(theta)
    dl = None if delta is None else _f64(delta)
    batch = X.reshape(-1, g.n)
    out = np.empty((batch.shape[0], g.m))
    for k in range(batch.shape[0]):
        xk = np.ascontiguousarray(batch[k])
        yk = np.empty(g.m)
        if g.fan_D is None:
            lib.orc_forward(g.N, g.B, g.V, _ptr(g.fov), _ptr(th), _ptr(dl), _ptr(xk), _ptr(yk))
        else:
            lib.orc_fan_forward(g.N, g.B, g.V, _ptr(g.fov), g.fan_D, _ptr(th), _ptr(dl), _ptr(xk), _ptr(yk))
        out[k] = yk
    return out.reshape(X.shape[:-1] + (g.m,)) if X.ndim > 1 else out[0]


def adjoint(g: Geometry, theta, Y, delta=None):
    """X = H(theta, delta)^T Y (scatter form).  Y: (V*B,) or (K, V*B)."""
    lib = _load()
    Y = _f64(Y)
    th = _f64(theta)
    dl = None if delta is None else _f64(delta)
    batch = Y.reshape(-1, g.m)
    out = np.empty((batch.shape[0], g.n))
    for k in range(batch.shape[0]):
        yk = np.ascontiguousarray(batch[k])
        xk = np.empty(g.n)
        if g.fan_D is None:
            lib.orc_adjoint(g.N, g.B, g.V, g.F, _ptr(g.fov), _ptr(th), _ptr(dl), _ptr(yk), _ptr(xk))
        else:
            lib.orc_fan_adjoint(g.N, g.B, g.V, g.F, _ptr(g.fov), g.fan_D, _ptr(th), _ptr(dl), _ptr(yk), _ptr(xk))
        out[k] = xk
    return out.reshape(Y.shape[:-1] + (g.n,)) if Y.ndim > 1 else out[0]


def dsample(g: Geometry, theta, X, delta=None):
    """Per-sample derivatives (d/dtheta_v, d/ddelta_v) of (H X)[v, b], each (V*B,)."""
    lib = _load()
    X = _f64(X)
    th = _f64(theta)
    dl = None if delta is None else _f64(delta)
    dt = np.empty(g.m)
    dd = np.empty(g.m)
    if g.fan_D is None:
        lib.orc_dsample(g.N, g.B, g.V, _ptr(g.fov), _ptr(th), _ptr(dl), _ptr(X), _ptr(dt), _ptr(dd))
    else:
        lib.orc_fan_dsample(g.N, g.B, g.V, _ptr(g.fov), g.fan_D, _ptr(th), _ptr(dl), _ptr(X), _ptr(dt), _ptr(dd))
    return dt, dd


def jac(g: Geometry, theta, X, dtheta, delta=None, ddelta=None):
    """dY = J_theta dtheta (+ J_delta ddelta)."""
    lib = _load()
    X, th, dth = _f64(X), _f64(theta), _f64(dtheta)
    dl = None if delta is None else _f64(delta)
    ddl = None if ddelta is None else _f64(ddelta)
    if g.fan_D is not None:  # per-sample derivatives times the per-view directions
        dt, dd = dsample(g, theta, X, delta)
        dy = (dt.reshape(g.V, g.B) * dth[:, None]).ravel()
        if ddl is not None:
            dy += (dd.reshape(g.V, g.B) * ddl[:, None]).ravel()
        return dy
    dy = np.empty(g.m)
    lib.orc_jac(g.N, g.B, g.V, _ptr(g.fov), _ptr(th), _ptr(dl), _ptr(X), _ptr(dth), _ptr(ddl), _ptr(dy))
    return dy


def jacT(g: Geometry, theta, X, R, delta=None):
    """(g_theta, g_delta) = (J_theta^T R, J_delta^T R), each (V,)."""
    lib = _load()
    X, th, R = _f64(X), _f64(theta), _f64(R)
    dl = None if delta is None else _f64(delta)
    if g.fan_D is not None:  # per-view sums of the residual times the per-sample derivatives
        dt, dd = dsample(g, theta, X, delta)
        return (dt * R).reshape(g.V, g.B).sum(1), (dd * R).reshape(g.V, g.B).sum(1)
    gt = np.empty(g.V)
    gd = np.empty(g.V)
    lib.orc_jacT(g.N, g.B, g.V, _ptr(g.fov), _ptr(th), _ptr(dl), _ptr(X), _ptr(R), _ptr(gt), _ptr(gd))
    return gt, gd


def dense_matrix(g: Geometry, theta, delta=None):
    """Assembled H (m x n) by applying the forward rule to unit vectors (small n only)."""
    if g.n > 4096:
        raise ValueError("dense assembly is for small images only")
    E = np.eye(g.n)
    return forward(g, theta, E, delta).T.copy()


def dense_adjoint_matrix(g: Geometry, theta, delta=None):
    """Assembled H^T (n x m) by applying the scatter adjoint to unit vectors."""
    if g.n * g.m > 64 * 1024 * 1024:
        raise ValueError("dense assembly is for small problems only")
    E = np.eye(g.m)
    return adjoint(g, theta, E, delta).T.copy()
