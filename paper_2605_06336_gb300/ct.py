"""Thin ctypes binding of libctgb.so (the C ABI in include/ctgb.h).

Functions carry the C names (``ct_init``, ``ct_forward``, ``ct_adjoint``,
``ct_jac``, ``ct_jacT``, ``ct_gn_terms``, ``ct_status``, ``ct_destroy``) and
only marshal arguments: tensors become device pointers, the current torch
stream becomes the handle's stream.  Every operator runs in the library's
CUDA kernels.  If the library is missing or no GPU is present the calls
raise; there is no fallback path.

:class:`CTOperator` bundles a handle with shape checks for torch tensors.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libctgb.so")

CT_OK = 0
CT_ERR_ARG = -1
CT_ERR_CUDA = -2
CT_ERR_OOM = -3
CT_ERR_TIMEOUT = -4
CT_ERR_NAN = -5
CT_ERR_NOCONV = -6


class CTError(RuntimeError):
    def __init__(self, code: int, what: str):
        lib = _lib_or_none()
        msg = lib.ct_strerror(code).decode() if lib else str(code)
        if code == CT_ERR_CUDA and lib:
            msg += " (" + lib.ct_last_cuda_error().decode() + ")"
        super().__init__(f"{what}: {msg}")
        self.code = code


class ct_geom(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32),
        ("B", ctypes.c_int32),
        ("n_views", ctypes.c_int32),
        ("n_frames", ctypes.c_int32),
        ("views_per_frame", ctypes.POINTER(ctypes.c_int32)),
        ("max_batch", ctypes.c_int32),
        ("use_offsets", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("source_distance", ctypes.c_double),
    ]


NLRMM_MAX_HIST = 256


class nlrmm_opts(ctypes.Structure):
    _fields_ = [
        ("k_min", ctypes.c_int32), ("k_max", ctypes.c_int32), ("outer_iters", ctypes.c_int32),
        ("maxiter_p", ctypes.c_int32), ("max_halvings", ctypes.c_int32), ("lam_iters", ctypes.c_int32),
        ("update_theta", ctypes.c_int32), ("stop_on_convergence", ctypes.c_int32),
        ("eps", ctypes.c_double), ("tol1", ctypes.c_double), ("tau", ctypes.c_double),
        ("noise_norm", ctypes.c_double), ("lam_fix", ctypes.c_double), ("lam_lo", ctypes.c_double),
        ("lam_hi", ctypes.c_double), ("c1", ctypes.c_double), ("beta", ctypes.c_double),
        ("alpha0", ctypes.c_double), ("mu_rel", ctypes.c_double), ("tol_u", ctypes.c_double),
        ("tol_p", ctypes.c_double), ("temporal", ctypes.c_int32), ("varpro", ctypes.c_int32),
        ("armijo_eps", ctypes.c_double), ("plain", ctypes.c_int32), ("shared_offset", ctypes.c_int32),
    ]


class nlrmm_stats(ctypes.Structure):
    _fields_ = [
        ("outer_done", ctypes.c_int32), ("converged", ctypes.c_int32), ("breakdown", ctypes.c_int32),
        ("enlarge_steps", ctypes.c_int32 * NLRMM_MAX_HIST),
        ("lambda_", ctypes.c_double * NLRMM_MAX_HIST), ("du", ctypes.c_double * NLRMM_MAX_HIST),
        ("dtheta", ctypes.c_double * NLRMM_MAX_HIST), ("rre", ctypes.c_double * NLRMM_MAX_HIST),
        ("ms", ctypes.c_double * NLRMM_MAX_HIST),
    ]


_lib = None


def _lib_or_none():
    return _lib


def load_library(path: str | None = None):
    """Open libctgb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2605_06336_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.ct_init.argtypes = [ctypes.POINTER(ct_geom), P, ctypes.POINTER(P)]
    lib.ct_destroy.argtypes = [P]
    lib.ct_destroy.restype = None
    lib.ct_forward.argtypes = [P, P, P, P, P, I]
    lib.ct_adjoint.argtypes = [P, P, P, P, P, I]
    lib.ct_forward_repeat.argtypes = [P, P, I]
    lib.ct_measure_peaks.argtypes = [P, P]
    lib.ct_measure_peaks.restype = ctypes.c_int
    lib.ct_adjoint_repeat.argtypes = [P, P, I]
    lib.ct_jac.argtypes = [P, P, P, P, P, P, P]
    lib.ct_jacT.argtypes = [P, P, P, P, P, P, P]
    lib.ct_gn_terms.argtypes = [P, P, P, P, P, P, P, P, P]
    lib.ct_jac_batch.argtypes = [P, P, P, P, P, P, P, I, I]
    lib.ct_jacT_batch.argtypes = [P, P, P, P, P, P, P, I, I]
    lib.ct_gn_terms_batch.argtypes = [P, P, P, P, P, P, P, P, P, I]
    lib.ct_status.argtypes = [P]
    lib.ct_set_stream.argtypes = [P, P]
    lib.ct_autotune.argtypes = [P]
    lib.ct_get_tuning.argtypes = [P, P]
    lib.ct_set_tuning.argtypes = [P, P]
    lib.ct_jacT_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P, P, P, P, P]
    lib.ct_jacT_noalloc.restype = ctypes.c_int
    lib.nlrmm_varpro.argtypes = [P, P, P, P, P, ctypes.c_int, ctypes.c_double, P, ctypes.c_double, P, P, P]
    lib.nlrmm_varpro.restype = ctypes.c_int
    lib.nlrmm_varpro_update.argtypes = [P, P, P, P, P, ctypes.c_int, ctypes.c_double, P, ctypes.c_double, P, P]
    lib.nlrmm_varpro_update.restype = ctypes.c_int
    lib.nlrmm_default_opts.argtypes = [P]
    lib.nlrmm_default_opts.restype = None
    lib.nlrmm_gks_solve.argtypes = [P, P, P, P, P, P, P, P]
    lib.nlrmm_gks_solve.restype = ctypes.c_int
    lib.nlrmm_stream_solve.argtypes = [P, ctypes.c_int, P, P, P, P, P, P, P, P]
    lib.nlrmm_stream_solve.restype = ctypes.c_int
    lib.ct_strerror.argtypes = [I]
    lib.ct_strerror.restype = ctypes.c_char_p
    lib.ct_last_cuda_error.argtypes = []
    lib.ct_last_cuda_error.restype = ctypes.c_char_p
    for f in ("ct_init", "ct_forward", "ct_adjoint", "ct_forward_repeat", "ct_adjoint_repeat", "ct_jac", "ct_jacT",
              "ct_gn_terms", "ct_jac_batch", "ct_jacT_batch", "ct_gn_terms_batch", "ct_status", "ct_set_stream",
              "ct_autotune", "ct_get_tuning", "ct_set_tuning"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != CT_OK:
        raise CTError(rc, what)


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# --- C-named entry points (argument marshalling only) ----------------------

def ct_init(N, B, n_views, views_per_frame=None, max_batch=1, precision=0, stream=None, source_distance=0.0):
    lib = load_library()
    g = ct_geom()
    g.N, g.B, g.n_views = int(N), int(B), int(n_views)
    keep = None
    if views_per_frame is not None:
        keep = (ctypes.c_int32 * len(views_per_frame))(*[int(v) for v in views_per_frame])
        g.n_frames = len(views_per_frame)
        g.views_per_frame = ctypes.cast(keep, ctypes.POINTER(ctypes.c_int32))
    else:
        g.n_frames = 1
        g.views_per_frame = None
    g.max_batch, g.use_offsets, g.precision = int(max_batch), 1, int(precision)
    g.source_distance = float(source_distance or 0.0)
    h = ctypes.c_void_p()
    _check(lib.ct_init(ctypes.byref(g), _stream_ptr(stream), ctypes.byref(h)), "ct_init")
    return h


def ct_destroy(h):
    load_library().ct_destroy(h)


def ct_forward(h, theta, delta, X, Y, batch):
    _check(load_library().ct_forward(h, _p(theta), _p(delta), _p(X), _p(Y), int(batch)), "ct_forward")


def ct_adjoint(h, theta, delta, Y, X, batch):
    _check(load_library().ct_adjoint(h, _p(theta), _p(delta), _p(Y), _p(X), int(batch)), "ct_adjoint")


def ct_measure_peaks():
    """(L2 read GB/s, shared-memory read GB/s) measured on the current device."""
    l2, sm = ctypes.c_double(), ctypes.c_double()
    _check(load_library().ct_measure_peaks(ctypes.byref(l2), ctypes.byref(sm)), "ct_measure_peaks")
    return l2.value, sm.value


def ct_forward_repeat(h, Y, batch):
    _check(load_library().ct_forward_repeat(h, _p(Y), int(batch)), "ct_forward_repeat")


def ct_adjoint_repeat(h, X, batch):
    _check(load_library().ct_adjoint_repeat(h, _p(X), int(batch)), "ct_adjoint_repeat")


def ct_jac(h, theta, delta, x, dtheta, ddelta, dy):
    _check(load_library().ct_jac(h, _p(theta), _p(delta), _p(x), _p(dtheta), _p(ddelta), _p(dy)), "ct_jac")


def ct_jacT(h, theta, delta, x, r, gtheta, gdelta):
    _check(load_library().ct_jacT(h, _p(theta), _p(delta), _p(x), _p(r), _p(gtheta), _p(gdelta)), "ct_jacT")


def ct_gn_terms(h, theta, delta, x, bdata, res, grad, jnorm2, fval):
    _check(load_library().ct_gn_terms(h, _p(theta), _p(delta), _p(x), _p(bdata), _p(res), _p(grad), _p(jnorm2),
                                      _p(fval)), "ct_gn_terms")


CT_BATCH_PER_IMAGE_DIRECTION, CT_BATCH_SHARED_R, CT_BATCH_SUM = 1, 2, 4


def ct_jac_batch(h, theta, delta, X, dtheta, ddelta, dY, batch, flags=0):
    _check(load_library().ct_jac_batch(h, _p(theta), _p(delta), _p(X), _p(dtheta), _p(ddelta), _p(dY), int(batch),
                                       int(flags)), "ct_jac_batch")


def ct_jacT_batch(h, theta, delta, X, R, gtheta, gdelta, batch, flags=0):
    _check(load_library().ct_jacT_batch(h, _p(theta), _p(delta), _p(X), _p(R), _p(gtheta), _p(gdelta), int(batch),
                                        int(flags)), "ct_jacT_batch")


def ct_gn_terms_batch(h, theta, delta, X, bdata, res, grad, jnorm2, fval, batch):
    _check(load_library().ct_gn_terms_batch(h, _p(theta), _p(delta), _p(X), _p(bdata), _p(res), _p(grad),
                                            _p(jnorm2), _p(fval), int(batch)), "ct_gn_terms_batch")


def ct_status(h):
    return load_library().ct_status(h)


def ct_set_stream(h, stream=None):
    _check(load_library().ct_set_stream(h, _stream_ptr(stream)), "ct_set_stream")


def ct_autotune(h):
    _check(load_library().ct_autotune(h), "ct_autotune")


TUNING_FIELDS = ("fwd_images_per_lane", "fwd_warps_per_ray", "fwd_views_per_cta", "adj_images_per_thread",
                 "adj_view_groups", "jac_warps_per_ray", "jac_views_per_cta", "fwd_staging", "jac_staging",
                 "adj_staging", "jac_images_per_lane", "fwd_interleaved")


def ct_get_tuning(h):
    buf = (ctypes.c_int32 * len(TUNING_FIELDS))()
    _check(load_library().ct_get_tuning(h, buf), "ct_get_tuning")
    return list(buf)


def ct_set_tuning(h, values):
    """The ct_set_tuning values in TUNING_FIELDS order; without the last one
    (fwd_interleaved) the forward reads the pair images."""
    values = list(values)
    if len(values) == len(TUNING_FIELDS) - 1:
        values.append(0)
    if len(values) != len(TUNING_FIELDS):
        raise ValueError(f"expected {len(TUNING_FIELDS)} launch-shape values, got {len(values)}")
    buf = (ctypes.c_int32 * len(TUNING_FIELDS))(*[int(v) for v in values])
    _check(load_library().ct_set_tuning(h, buf), "ct_set_tuning")


NOALLOC_MAX_N, NOALLOC_MAX_VIEWS, NOALLOC_MAX_BINS = 256, 512, 1024


def _noalloc_args(specs):
    """Check the tensor arguments of ct_jacT_noalloc (the C entry point reads and
    writes through raw pointers with the sizes it is given): specs are
    (name, tensor or None, dtype, element count, required).  Types, counts and
    strides of every argument are checked before any device."""
    import torch
    for name, t, dtype, numel, required in specs:
        if t is None:
            if required:
                raise ValueError(f"ct_jacT_noalloc: {name} is required")
            continue
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"ct_jacT_noalloc: {name} must be a torch tensor")
        if t.dtype != dtype:
            raise ValueError(f"ct_jacT_noalloc: {name} must be {dtype}, got {t.dtype}")
        if t.numel() != numel:
            raise ValueError(f"ct_jacT_noalloc: {name} must have {numel} elements, got {t.numel()}")
        if not t.is_contiguous():
            raise ValueError(f"ct_jacT_noalloc: {name} must be contiguous")
    for name, t, _, _, _ in specs:
        if t is not None and not t.is_cuda:
            raise ValueError(f"ct_jacT_noalloc: {name} must be a CUDA tensor")


def ct_jacT_noalloc(N, B, n_views, theta, delta, x, r, gtheta, gdelta, stream=None):
    """ct_jacT without a handle or any device allocation (for callers that cannot
    allocate); the workspace is a static device array, so sizes are capped.
    theta, delta (or None), gtheta, gdelta (or None): float64 [n_views]; x:
    float32 [N*N]; r: float32 [n_views*B]; all contiguous CUDA tensors."""
    import torch
    N, B, n_views = int(N), int(B), int(n_views)
    if N < 2 or B < 1 or n_views < 1:
        raise ValueError(f"ct_jacT_noalloc: N={N}, B={B}, views={n_views} below the minimum 2/1/1")
    if N > NOALLOC_MAX_N or B > NOALLOC_MAX_BINS or n_views > NOALLOC_MAX_VIEWS:
        raise ValueError(f"ct_jacT_noalloc: N={N}, B={B}, views={n_views} exceed the limits "
                         f"{NOALLOC_MAX_N}/{NOALLOC_MAX_BINS}/{NOALLOC_MAX_VIEWS} of its static workspace")
    _noalloc_args([("theta", theta, torch.float64, n_views, True), ("delta", delta, torch.float64, n_views, False),
                   ("x", x, torch.float32, N * N, True), ("r", r, torch.float32, n_views * B, True),
                   ("gtheta", gtheta, torch.float64, n_views, True),
                   ("gdelta", gdelta, torch.float64, n_views, False)])
    _check(load_library().ct_jacT_noalloc(int(N), int(B), int(n_views), _p(theta), _p(delta), _p(x), _p(r),
                                          _p(gtheta), _p(gdelta), _stream_ptr(stream)), "ct_jacT_noalloc")


def nlrmm_default_opts(**overrides):
    o = nlrmm_opts()
    load_library().nlrmm_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def nlrmm_gks_solve(h, b, theta_inout, delta, x_out, x_true=None, opts=None, **overrides):
    """Run the GPU NL-RMM-GKS driver; returns (status code, stats dict)."""
    o = opts if opts is not None else nlrmm_default_opts(**overrides)
    st = nlrmm_stats()
    rc = load_library().nlrmm_gks_solve(h, _p(b), _p(theta_inout), _p(delta), _p(x_out), _p(x_true),
                                        ctypes.byref(o), ctypes.byref(st))
    if rc not in (CT_OK, CT_ERR_NOCONV):
        raise CTError(rc, "nlrmm_gks_solve")
    k = min(st.outer_done, NLRMM_MAX_HIST)
    stats = {"rc": rc, "outer_done": st.outer_done, "converged": bool(st.converged), "breakdown": bool(st.breakdown),
             "enlarge_steps": list(st.enlarge_steps[:k]), "lambda": list(st.lambda_[:k]), "du": list(st.du[:k]),
             "dtheta": list(st.dtheta[:k]), "rre": list(st.rre[:k]), "ms": list(st.ms[:k])}
    return rc, stats


def nlrmm_stream_solve(handles, bs, thetas, deltas, noise_norms, x_out, x_true=None, opts=None, **overrides):
    """Run the GPU streaming NL-RMM-GKS over blocks; returns (status code, stats dict per pass)."""
    o = opts if opts is not None else nlrmm_default_opts(**overrides)
    nb = len(handles)
    if not (len(bs) == len(thetas) == nb) or (deltas is not None and len(deltas) != nb):
        raise ValueError("one data vector, angle vector (and offset vector) per block")
    Parr = ctypes.c_void_p * nb
    hs = Parr(*[h for h in handles])
    barr = Parr(*[_p(b) for b in bs])
    tharr = Parr(*[_p(t) for t in thetas])
    darr = None if deltas is None else Parr(*[_p(d) for d in deltas])
    narr = None if noise_norms is None else (ctypes.c_double * nb)(*[float(x) for x in noise_norms])
    st = nlrmm_stats()
    rc = load_library().nlrmm_stream_solve(hs, nb, barr, tharr, darr, narr, _p(x_out), _p(x_true),
                                           ctypes.byref(o), ctypes.byref(st))
    if rc not in (CT_OK, CT_ERR_NOCONV):
        raise CTError(rc, "nlrmm_stream_solve")
    k = min(st.outer_done, NLRMM_MAX_HIST)
    stats = {"rc": rc, "passes": st.outer_done, "converged": bool(st.converged), "breakdown": bool(st.breakdown),
             "enlarge_steps": list(st.enlarge_steps[:k]), "lambda": list(st.lambda_[:k]), "du": list(st.du[:k]),
             "dtheta": list(st.dtheta[:k]), "rre": list(st.rre[:k]), "ms": list(st.ms[:k])}
    return rc, stats


def stream_solve(ops, bs, thetas0, noise_norms, deltas=None, x_true=None, **opts):
    """Streaming NL-RMM-GKS over blocks (one CTOperator per block, sharing the
    image size): returns (x, thetas, stats).  thetas0 are not modified."""
    op0 = ops[0]
    for op, b in zip(ops, bs):
        op._chk(b, op.m, "b")
    thetas = [op._ang(t, "theta0").clone() for op, t in zip(ops, thetas0)]
    dl = None if deltas is None else [op._ang(d, "delta") for op, d in zip(ops, deltas)]
    x = torch.empty(op0.n, dtype=op0.dtype, device=bs[0].device)
    if x_true is not None:
        op0._chk(x_true, op0.n, "x_true")
    _, stats = nlrmm_stream_solve([op.h for op in ops], bs, thetas, dl, noise_norms, x, x_true, **opts)
    return x, thetas, stats


def nlrmm_varpro(h, b, theta, delta, V, k, lam, u_w, eps, fval, grad=None, u_out=None):
    _check(load_library().nlrmm_varpro(h, _p(b), _p(theta), _p(delta), _p(V), int(k), float(lam), _p(u_w),
                                       float(eps), _p(fval), _p(grad), _p(u_out)), "nlrmm_varpro")


def nlrmm_varpro_update(h, b, theta_inout, delta, V, k, lam, u_w, eps, opts=None, **overrides):
    """One VarPro parameter update (theta_inout updated in place); returns the
    reduced objective before the first step and after each step."""
    o = opts if opts is not None else nlrmm_default_opts(**overrides)
    f_hist = (ctypes.c_double * (max(o.maxiter_p, 0) + 1))()
    _check(load_library().nlrmm_varpro_update(h, _p(b), _p(theta_inout), _p(delta), _p(V), int(k), float(lam),
                                              _p(u_w), float(eps), ctypes.byref(o), f_hist),
           "nlrmm_varpro_update")
    return list(f_hist)


# --- tensor-level wrapper ---------------------------------------------------

class CTOperator:
    """A ct handle plus shape/dtype checks for CUDA tensors.

    Images are ``(K, F*N*N)`` (or ``(F*N*N,)``), sinograms ``(K, V*B)``;
    angles/offsets are float64 CUDA tensors of length V.
    """

    def __init__(self, N, B, n_views, views_per_frame=None, max_batch=8, dtype=torch.float32, device="cuda",
                 source_distance=None):
        """source_distance: None for the parallel beam, else the fan-beam source
        distance from the rotation centre in pixels (see ct_geom)."""
        if dtype not in (torch.float32, torch.float64):
            raise ValueError("dtype must be float32 or float64")
        self.N, self.B, self.V = int(N), int(B), int(n_views)
        self.views_per_frame = list(views_per_frame) if views_per_frame is not None else [self.V]
        self.F = len(self.views_per_frame)
        self.max_batch = int(max_batch)
        self.dtype = dtype
        self.device = torch.device(device)
        self.source_distance = source_distance
        with torch.cuda.device(self.device):
            self.h = ct_init(N, B, n_views, views_per_frame, max_batch, 1 if dtype == torch.float64 else 0,
                             source_distance=source_distance or 0.0)

    @property
    def n(self):
        return self.F * self.N * self.N

    @property
    def m(self):
        return self.V * self.B

    def close(self):
        if getattr(self, "h", None) is not None:
            ct_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, t, last, name):
        if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous() and t.shape[-1] == last):
            raise ValueError(f"{name}: expected contiguous {self.dtype} CUDA tensor with last dim {last}, "
                             f"got {tuple(t.shape)} {t.dtype} {t.device}")

    def _ang(self, a, name):
        if a is None:
            return None
        if not (a.is_cuda and a.dtype == torch.float64 and a.is_contiguous() and a.numel() == self.V):
            raise ValueError(f"{name}: expected contiguous float64 CUDA tensor of {self.V} views")
        return a

    def forward(self, X, theta, delta=None, out=None, batch=None):
        """Y = H(theta, delta) X.  X = None: the images of the previous call on this
        operator that took images (their layouts are reused), `batch` of them (1
        by default)."""
        if X is None:
            K = int(batch or 1)
            shape = (self.m,) if batch is None else (K, self.m)
            dev = theta.device
        else:
            self._chk(X, self.n, "X")
            K = 1 if X.dim() == 1 else X.shape[0]
            shape, dev = X.shape[:-1] + (self.m,), X.device
        Y = out if out is not None else torch.empty(shape, dtype=self.dtype, device=dev)
        ct_forward(self.h, self._ang(theta, "theta"), self._ang(delta, "delta"), X, Y, K)
        return Y

    def adjoint(self, Y, theta, delta=None, out=None):
        self._chk(Y, self.m, "Y")
        K = 1 if Y.dim() == 1 else Y.shape[0]
        X = out if out is not None else torch.empty(Y.shape[:-1] + (self.n,), dtype=self.dtype, device=Y.device)
        ct_adjoint(self.h, self._ang(theta, "theta"), self._ang(delta, "delta"), Y, X, K)
        return X

    def _img(self, x, name):
        """x, checked; None (the image of the previous call that took one) passes."""
        if x is not None:
            self._chk(x, self.n, name)
        return x

    def jac(self, x, theta, dtheta, delta=None, ddelta=None, out=None):
        self._img(x, "x")
        dy = out if out is not None else torch.empty(self.m, dtype=self.dtype, device=theta.device)
        ct_jac(self.h, self._ang(theta, "theta"), self._ang(delta, "delta"), x, self._ang(dtheta, "dtheta"),
               self._ang(ddelta, "ddelta"), dy)
        return dy

    def jacT(self, x, theta, r, delta=None, want_delta=False):
        self._img(x, "x")
        self._chk(r, self.m, "r")
        gt = torch.empty(self.V, dtype=torch.float64, device=r.device)
        gd = torch.empty(self.V, dtype=torch.float64, device=r.device) if want_delta else None
        ct_jacT(self.h, self._ang(theta, "theta"), self._ang(delta, "delta"), x, r, gt, gd)
        return (gt, gd) if want_delta else gt

    def _batch(self, X, last, name):
        self._chk(X, last, name)
        K = 1 if X.dim() == 1 else X.shape[0]
        if K > self.max_batch:
            raise ValueError(f"{name}: batch {K} above max_batch {self.max_batch}")
        return K

    def jac_batch(self, X, theta, dtheta, delta=None, ddelta=None, out=None):
        """dY[k] = J(x_k) dtheta (+ J_delta(x_k) ddelta) for the K images of X in one
        launch; dtheta / ddelta are [V] (shared) or [K, V] (one per image)."""
        K = self._batch(X, self.n, "X")
        per = dtheta.dim() == 2
        for nm, d in (("dtheta", dtheta), ("ddelta", ddelta)):
            if d is not None and not (d.is_cuda and d.dtype == torch.float64 and d.is_contiguous() and
                                      d.numel() == (K * self.V if per else self.V)):
                raise ValueError(f"{nm}: expected contiguous float64 CUDA tensor of {K if per else 1} x {self.V}")
        dY = out if out is not None else torch.empty(X.shape[:-1] + (self.m,), dtype=self.dtype, device=X.device)
        ct_jac_batch(self.h, self._ang(theta, "theta"), self._ang(delta, "delta"), X, dtheta, ddelta, dY, K,
                     CT_BATCH_PER_IMAGE_DIRECTION if per else 0)
        return dY

    def jacT_batch(self, X, theta, R, delta=None, want_delta=False, sum_images=False):
        """g[k] = J(x_k)^T R_k for the K images of X in one launch; R is [K, m] or
        one [m] sinogram shared by every image.  sum_images: one [V] gradient,
        the images added in order."""
        K = self._batch(X, self.n, "X")
        self._chk(R, self.m, "R")
        shared = R.dim() == 1
        if not shared and R.shape[0] != K:
            raise ValueError(f"R: {R.shape[0]} sinograms for {K} images")
        shape = (self.V,) if sum_images else (K, self.V)
        gt = torch.empty(shape, dtype=torch.float64, device=X.device)
        gd = torch.empty(shape, dtype=torch.float64, device=X.device) if want_delta else None
        flags = (CT_BATCH_SHARED_R if shared else 0) | (CT_BATCH_SUM if sum_images else 0)
        ct_jacT_batch(self.h, self._ang(theta, "theta"), self._ang(delta, "delta"), X, R, gt, gd, K, flags)
        return (gt, gd) if want_delta else gt

    def gn_terms_batch(self, X, theta, bdata, delta=None, want_residual=False):
        """ct_gn_terms for each of the K images of X against the K data sinograms bdata."""
        K = self._batch(X, self.n, "X")
        self._chk(bdata, self.m, "bdata")
        if (1 if bdata.dim() == 1 else bdata.shape[0]) != K:
            raise ValueError("bdata: one data sinogram per image expected")
        res = torch.empty((K, self.m), dtype=self.dtype, device=X.device) if want_residual else None
        g, j2, f = (torch.empty((K, self.V), dtype=torch.float64, device=X.device) for _ in range(3))
        ct_gn_terms_batch(self.h, self._ang(theta, "theta"), self._ang(delta, "delta"), X, bdata, res, g, j2, f, K)
        return g, j2, f, res

    def gn_terms(self, x, theta, bdata, delta=None, want_residual=False):
        self._img(x, "x")
        self._chk(bdata, self.m, "bdata")
        res = torch.empty(self.m, dtype=self.dtype, device=bdata.device) if want_residual else None
        g = torch.empty(self.V, dtype=torch.float64, device=bdata.device)
        j2 = torch.empty(self.V, dtype=torch.float64, device=bdata.device)
        f = torch.empty(self.V, dtype=torch.float64, device=bdata.device)
        ct_gn_terms(self.h, self._ang(theta, "theta"), self._ang(delta, "delta"), x, bdata, res, g, j2, f)
        return g, j2, f, res

    def status(self):
        return ct_status(self.h)

    def autotune(self):
        ct_autotune(self.h)
        return ct_get_tuning(self.h)

    @property
    def tuning(self):
        return ct_get_tuning(self.h)

    @tuning.setter
    def tuning(self, values):
        ct_set_tuning(self.h, values)

    def set_stream(self, stream=None):
        ct_set_stream(self.h, stream)

    def varpro(self, b, theta, V, lam, u_w=None, eps=1e-3, delta=None, want_grad=True):
        """VarPro reduced objective on the basis V (k x n): returns (f, grad or None, u)."""
        self._chk(b, self.m, "b")
        self._chk(V, self.n, "V")
        fval = torch.empty(1, dtype=torch.float64, device=b.device)
        grad = torch.empty(self.V, dtype=torch.float64, device=b.device) if want_grad else None
        u = torch.empty(self.n, dtype=self.dtype, device=b.device)
        if u_w is not None:
            self._chk(u_w, self.n, "u_w")
        nlrmm_varpro(self.h, b, self._ang(theta, "theta"), self._ang(delta, "delta"), V.contiguous(),
                     V.shape[0], lam, u_w, eps, fval, grad, u)
        return fval[0], grad, u

    def varpro_update(self, b, theta, V, lam, u_w=None, eps=1e-3, delta=None, **opts):
        """VarPro Gauss-Newton update of the angles on the basis V (k x n):
        returns (new angles, reduced objective per step).  theta is not modified."""
        self._chk(b, self.m, "b")
        self._chk(V, self.n, "V")
        if u_w is not None:
            self._chk(u_w, self.n, "u_w")
        th = self._ang(theta, "theta").clone()
        f_hist = nlrmm_varpro_update(self.h, b, th, self._ang(delta, "delta"), V.contiguous(), V.shape[0], lam,
                                     u_w, eps, **opts)
        return th, f_hist

    def solve(self, b, theta0, delta=None, x_true=None, **opts):
        """NL-RMM-GKS: returns (x, theta, stats).  theta0 is not modified."""
        self._chk(b, self.m, "b")
        theta = self._ang(theta0, "theta0").clone()
        x = torch.empty(self.n, dtype=self.dtype, device=b.device)
        if x_true is not None:
            self._chk(x_true, self.n, "x_true")
        _, stats = nlrmm_gks_solve(self.h, b, theta, self._ang(delta, "delta"), x, x_true, **opts)
        return x, theta, stats
