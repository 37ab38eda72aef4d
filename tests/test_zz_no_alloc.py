"""The allocation-free entry point ct_jacT_noalloc, through the C ABI.

Some callers cannot allocate device memory (a host application that owns all
of it through its own pool, a service whose budget is fixed after start-up);
ct_jacT_noalloc serves them with a static device workspace.  Its results must
equal those of ct_jacT, the entry point it mirrors, and the FP64 oracle's, on
calls in a row: the
second call keeps the first call's angles and offsets but changes the image
size and the bin count, so a per-view table left over from the first call
(its constants are cached by angle and offset) would give wrong gradients;
a third call passes no offsets.  A non-finite angle makes that view's outputs
NaN.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2605_06336_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _rel(a, b):
    return float((a - b).norm() / b.norm())


def test_noalloc_matches_ct_jacT_on_calls_in_a_row():
    from paper_2605_06336_gb300 import ct
    ct.load_library()
    rng = np.random.default_rng(1)
    V = 60
    theta = _dev(synth.random_angles(V, rng), torch.float64)
    delta = _dev(rng.normal(0, 0.5, V), torch.float64)
    # same angles and offsets, other geometry; then the same geometry without offsets
    for N, with_delta in ((64, True), (200, True), (200, False)):
        B = synth.n_bins(N)
        x = _dev(rng.uniform(size=N * N), torch.float32)
        r = _dev(rng.standard_normal(V * B), torch.float32)
        dl = delta if with_delta else None
        op = ct.CTOperator(N, B, V, max_batch=1, dtype=torch.float32)
        if with_delta:
            gt_ref, gd_ref = op.jacT(x, theta, r, dl, want_delta=True)
        else:
            gt_ref = op.jacT(x, theta, r)
        gt = torch.full((V,), float("nan"), dtype=torch.float64, device="cuda")
        gd = torch.full((V,), float("nan"), dtype=torch.float64, device="cuda") if with_delta else None
        ct.ct_jacT_noalloc(N, B, V, theta, dl, x, r, gt, gd)
        torch.cuda.synchronize()
        assert _rel(gt, gt_ref) <= 1e-5, (N, with_delta)
        if with_delta:
            assert _rel(gd, gd_ref) <= 1e-5, N
        # and against the FP64 oracle directly, so a defect shared with ct_jacT would show
        g = oracle.Geometry(N, B, V)
        d_h = delta.cpu().numpy() if with_delta else None
        gto, gdo = oracle.jacT(g, theta.cpu().numpy(), x.double().cpu().numpy(), r.double().cpu().numpy(), d_h)
        assert np.linalg.norm(gt.cpu().numpy() - gto) <= 1e-5 * np.linalg.norm(gto), (N, with_delta)
        if with_delta:
            assert np.linalg.norm(gd.cpu().numpy() - gdo) <= 1e-5 * np.linalg.norm(gdo), N
        op.close()


def test_noalloc_marks_views_with_non_finite_angles():
    from paper_2605_06336_gb300 import ct
    rng = np.random.default_rng(2)
    N, V = 32, 12
    B = synth.n_bins(N)
    th = synth.random_angles(V, rng)
    th[3] = np.nan
    dl = rng.normal(0, 0.5, V)
    dl[7] = np.inf
    gt = torch.zeros(V, dtype=torch.float64, device="cuda")
    gd = torch.zeros(V, dtype=torch.float64, device="cuda")
    ct.ct_jacT_noalloc(N, B, V, _dev(th, torch.float64), _dev(dl, torch.float64),
                       _dev(rng.uniform(size=N * N), torch.float32), _dev(rng.standard_normal(V * B), torch.float32),
                       gt, gd)
    torch.cuda.synchronize()
    bad = np.zeros(V, bool)
    bad[[3, 7]] = True
    assert np.all(np.isnan(gt.cpu().numpy()[bad])) and np.all(np.isnan(gd.cpu().numpy()[bad]))
    assert np.all(np.isfinite(gt.cpu().numpy()[~bad])) and np.all(np.isfinite(gd.cpu().numpy()[~bad]))


def test_noalloc_rejects_sizes_beyond_its_workspace():
    from paper_2605_06336_gb300 import ct
    lib = ct.load_library()
    rc = lib.ct_jacT_noalloc(ct.NOALLOC_MAX_N + 1, 8, 4, ctypes.c_void_p(1), None, ctypes.c_void_p(1),
                             ctypes.c_void_p(1), ctypes.c_void_p(1), None, None)
    assert rc == ct.CT_ERR_ARG
    with pytest.raises(ValueError):
        ct.ct_jacT_noalloc(ct.NOALLOC_MAX_N + 1, 8, 4, None, None, None, None, None, None)
