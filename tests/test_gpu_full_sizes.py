"""Parity at the full sizes of the remaining workloads, at autotuned launch shapes.

* 512^2 image, 360 views with angle errors and per-view detector offsets,
  725 bins: H, H^T, J (angle and offset directions) and J^T (both gradients)
  against the FP64 oracle, and the autograd Function's directional
  derivatives against central differences of the FP64 GPU forward on 32
  random directions (h = 1e-4, 1e-5, 1e-6; interpolation kinks make the
  quotient inexact, by an error that shrinks with h).
* 16 frames of 256^2 with 30-120 golden-angle views each, 363 bins: H and
  H^T on a 2-image batch of all frames, J and J^T on one.
* One 120-view chunk of the 2048^2 / 1440-view grid (angle errors
  N(0, 0.25 deg^2)), 2897 bins: H, H^T, J and J^T.
The oracle computes every output (plain C, FP64, seconds per operator at these
sizes); the images of the batch beyond the phantom are uniform random, as the
operators are linear in them.  Each bound holds normwise and element by
element: per view for sinograms (max |error| / max |oracle| of the view), per
image row for images, and per view for J^T against the magnitude of the terms
its sum over bins adds up, so that an error confined to a few samples (one
flipped interpolation cell at 2048^2) is not averaged away.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_06336_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def rows_rel(a, b, ncols):
    a = np.asarray(a, dtype=np.float64).reshape(-1, ncols)
    b = np.asarray(b, dtype=np.float64).reshape(-1, ncols)
    scale = np.abs(b).max(1)
    scale[scale == 0] = 1.0
    return float((np.abs(a - b).max(1) / scale).max())


def view_sum_rel(gv, go, r, dt, V, B):
    mag = (np.abs(np.asarray(r).reshape(V, B)) * np.abs(np.asarray(dt).reshape(V, B))).sum(1)
    mag[mag == 0] = 1.0
    return float((np.abs(np.asarray(gv) - np.asarray(go)) / mag).max())


def _check_all(op, g, theta, delta, X, rng, tol=1e-5):
    """H, H^T on the batch, J / J^T on its first image, against the oracle."""
    V, B, N = g.V, g.B, g.N
    th = dev(theta)
    dl = None if delta is None else dev(delta)
    Y = host(op.forward(dev(X, torch.float32), th, dl))
    Yo = oracle.forward(g, theta, X, delta)
    assert rel(Y, Yo) <= tol
    assert rows_rel(Y, Yo, B) <= tol
    R = rng.standard_normal(Yo.shape)
    Xa = host(op.adjoint(dev(R, torch.float32), th, dl))
    Xo = oracle.adjoint(g, theta, R, delta)
    assert rel(Xa, Xo) <= tol
    assert rows_rel(Xa, Xo, N) <= tol
    dth = rng.standard_normal(V)
    ddl = None if delta is None else rng.standard_normal(V)
    dy = host(op.jac(dev(X[0], torch.float32), th, dev(dth), dl, None if ddl is None else dev(ddl)))
    dyo = oracle.jac(g, theta, X[0], dth, delta, ddl)
    assert rel(dy, dyo) <= tol
    assert rows_rel(dy, dyo, B) <= tol
    r = R[0]
    gt_o, gd_o = oracle.jacT(g, theta, X[0], r, delta)
    dt, dd = oracle.dsample(g, theta, X[0], delta)
    if delta is None:
        gt = host(op.jacT(dev(X[0], torch.float32), th, dev(r, torch.float32)))
    else:
        gt, gd = op.jacT(dev(X[0], torch.float32), th, dev(r, torch.float32), dl, want_delta=True)
        gt = host(gt)
        assert rel(host(gd), gd_o) <= tol
        assert view_sum_rel(host(gd), gd_o, r, dd, V, B) <= tol
    assert rel(gt, gt_o) <= tol
    assert view_sum_rel(gt, gt_o, r, dt, V, B) <= tol


def test_512_image_360_views_with_offsets():
    from paper_2605_06336_gb300 import ct
    w = synth.make_workload("C3")
    rng = np.random.default_rng(41)
    X = np.stack([w.images.reshape(-1), rng.uniform(size=w.N * w.N)])
    op = ct.CTOperator(w.N, w.B, w.V, max_batch=2, dtype=torch.float32)
    op.autotune()
    _check_all(op, oracle.Geometry(w.N, w.B, w.V), w.theta_true, w.delta_true, X, rng)


def test_512_image_autograd_central_differences():
    from paper_2605_06336_gb300.autograd import project
    from paper_2605_06336_gb300 import ct
    w = synth.make_workload("C3")
    op = ct.CTOperator(w.N, w.B, w.V, max_batch=1, dtype=torch.float64)
    rng = np.random.default_rng(42)
    x = dev(w.images.reshape(-1))
    th0, dl0 = dev(w.theta_true), dev(w.delta_true)
    wt = dev(rng.standard_normal(w.V * w.B))
    th = th0.clone().requires_grad_(True)
    dl = dl0.clone().requires_grad_(True)
    (project(x, th, op, dl) * wt).sum().backward()
    dirs = [(dev(rng.standard_normal(w.V)), dev(rng.standard_normal(w.V))) for _ in range(32)]
    errs = {}
    for h in (1e-4, 1e-5, 1e-6):
        err = ref = 0.0
        for dth, ddl in dirs:
            lp = float((op.forward(x, th0 + h * dth, dl0 + h * ddl) * wt).sum())
            lm = float((op.forward(x, th0 - h * dth, dl0 - h * ddl) * wt).sum())
            an = float((th.grad * dth).sum() + (dl.grad * ddl).sum())
            err += abs((lp - lm) / (2 * h) - an)
            ref += abs(an)
        errs[h] = err / ref
    # Each (ray, row) step whose interpolation cell changes inside [-h, h] adds
    # an error of either sign; at this size ~1e8 steps contribute, so the sum
    # shrinks like sqrt(h) (a factor ~3.2 per decade) rather than like h.
    assert errs[1e-4] <= 5e-2, errs
    assert errs[1e-5] <= errs[1e-4] / 2.5 and errs[1e-6] <= errs[1e-5] / 2.5, errs
    assert errs[1e-6] <= 5e-3, errs


def test_16_frames_golden_angle_views():
    from paper_2605_06336_gb300 import ct
    w = synth.make_workload("C4")
    rng = np.random.default_rng(43)
    n = w.F * w.N * w.N
    X = np.stack([w.images.reshape(-1), rng.uniform(size=n)])
    op = ct.CTOperator(w.N, w.B, w.V, w.views_per_frame, max_batch=2, dtype=torch.float32)
    op.autotune()
    _check_all(op, oracle.Geometry(w.N, w.B, w.V, w.views_per_frame), w.theta_true, None, X, rng)


def test_2048_image_one_120_view_chunk():
    from paper_2605_06336_gb300 import ct
    N, V_all = 2048, 1440
    B = synth.n_bins(N)
    rng = np.random.default_rng(44)
    nominal = np.arange(V_all) * (math.pi / V_all)
    theta_all = nominal + rng.normal(0.0, 0.5 * math.pi / 180.0, V_all)  # sigma = 0.5 deg: N(0, 0.25 deg^2)
    chunk = np.sort(rng.permutation(V_all)[:120])
    theta = theta_all[chunk]
    X = rng.uniform(size=(1, N * N))
    op = ct.CTOperator(N, B, 120, max_batch=1, dtype=torch.float32)
    op.autotune()
    _check_all(op, oracle.Geometry(N, B, 120), theta, None, X, rng)


@pytest.mark.parametrize("size", ["512", "2048"])
def test_interleaved_forward_at_full_sizes(size):
    """The forward on images interleaved in groups of 4 (the layout the benchmark's
    autotuned runs pick at these sizes) at the 512^2 / 360-view workload with offsets
    and on a 120-view chunk of the 2048^2 grid: the same bits as on the pair images
    for a batch of 5 (one group of 4 and one single image), and the phantom's
    sinogram within the FP32 bound of the oracle, per view."""
    from paper_2605_06336_gb300 import ct
    rng = np.random.default_rng(45)
    if size == "512":
        w = synth.make_workload("C3")
        N, B, V, theta, delta = w.N, w.B, w.V, w.theta_true, w.delta_true
        x0 = w.images.reshape(-1)
    else:
        N, V = 2048, 120
        B = synth.n_bins(N)
        theta = np.sort(rng.uniform(0.0, math.pi, V))
        delta = None
        x0 = rng.uniform(size=N * N)
    X = np.stack([x0] + [rng.uniform(size=N * N) for _ in range(4)])
    th = dev(theta)
    dl = None if delta is None else dev(delta)
    Xg = dev(X, torch.float32)
    out = []
    for layout in (0, 1):
        op = ct.CTOperator(N, B, V, max_batch=5, dtype=torch.float32)
        op.tuning = [4, 4, 1, 4, 2, 4, 1, 0, 0, 0, 1, layout]
        out.append(op.forward(Xg, th, dl).clone())
        op.close()
    assert torch.equal(out[0], out[1])
    y = host(out[1][0])
    yo = oracle.forward(oracle.Geometry(N, B, V), theta, x0, delta)
    assert rel(y, yo) <= 1e-5 and rows_rel(y, yo, B) <= 1e-5
