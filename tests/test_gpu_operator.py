"""GPU parity: the CUDA operators (through the C ABI) against the FP64 oracle.

Tolerances (normwise relative, ||gpu - oracle|| / ||oracle||):
  * float32 operators: 1e-5 for H, H^T, J and J^T;
  * float64 operators: 1e-12.
The same bounds hold element by element, so that an error confined to a few
samples (one flipped interpolation cell) is not averaged away: per view for
sinograms, max_b |gpu - oracle| / max_b |oracle|; per image row for images;
per view for J^T, |gpu - oracle| / sum_b |r_vb| |dH x/dtheta_v|_b (the
magnitude of the terms the view's sum cancels).
Angles are kept away from |cos| = |sin| (the Joseph axis switch), where the
two sides could break the tie differently in the last bit.  For the angle
derivative the view at "pi/2" is pi/2 + 1e-7: at pi/2 itself cos() is 6e-17,
a ray slope below the 2^-49 resolution of the kernels' fixed-point line, and
the one-sided slope chosen at the (then exact) interpolation kinks depends on
the sign of that sub-resolution slope.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_06336_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float32: 1e-5, torch.float64: 1e-12}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def rows_rel(a, b, ncols):
    """max over rows of max|a - b| / max|b| in that row (rows of ncols entries;
    rows of b that are all zero are compared against 1)."""
    a = np.asarray(a, dtype=np.float64).reshape(-1, ncols)
    b = np.asarray(b, dtype=np.float64).reshape(-1, ncols)
    if a.size == 0:
        return 0.0
    scale = np.abs(b).max(1)
    scale[scale == 0] = 1.0
    return float((np.abs(a - b).max(1) / scale).max())


def view_sum_rel(gv, go, r, dt, V, B):
    """per-view error of a sum over bins, against the magnitude of its terms"""
    mag = (np.abs(np.asarray(r).reshape(V, B)) * np.abs(np.asarray(dt).reshape(V, B))).sum(1)
    mag[mag == 0] = 1.0
    return float((np.abs(np.asarray(gv) - np.asarray(go)) / mag).max()) if V else 0.0


@pytest.fixture(scope="module")
def ct():
    from paper_2605_06336_gb300 import ct as ctmod
    ctmod.load_library()
    return ctmod


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


CASES = [
    # (N, B, views_per_frame, batch, offsets)
    (2, 3, [5], 1, False),
    (16, 23, [8], 3, True),
    (37, 53, [11], 11, False),       # ragged tiles, ragged warps, batch 8+2+1
    (24, 35, [4, 1, 0, 6], 2, True),  # uneven frames, one empty
    (64, 91, [90], 8, False),         # small end-to-end workload shape
]


def _case_inputs(N, B, vpf, batch, offs, seed, near_axis=0.0):
    rng = np.random.default_rng(seed)
    V = sum(vpf)
    theta = synth.random_angles(V, rng)
    if V >= 3:
        theta[0], theta[1] = 0.0, math.pi / 2 + near_axis  # axis-aligned views
    delta = rng.normal(0, 0.5, V) if offs else None
    F = len(vpf)
    X = rng.uniform(size=(batch, F * N * N))
    Y = rng.standard_normal((batch, V * B))
    return theta, delta, X, Y


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("case", CASES)
def test_forward_adjoint_parity(ct, case, dtype):
    N, B, vpf, batch, offs = case
    theta, delta, X, Y = _case_inputs(N, B, vpf, batch, offs, seed=N * 7 + batch)
    g = oracle.Geometry(N, B, sum(vpf), vpf)
    op = ct.CTOperator(N, B, sum(vpf), vpf, max_batch=batch, dtype=dtype)
    th, dl = dev(theta), (dev(delta) if delta is not None else None)
    Yg = op.forward(dev(X, dtype), th, dl)
    Xg = op.adjoint(dev(Y, dtype), th, dl)
    torch.cuda.synchronize()
    assert op.status() == ct.CT_OK
    Yo = oracle.forward(g, theta, X, delta)
    Xo = oracle.adjoint(g, theta, Y, delta)
    assert rel(host(Yg), Yo) <= TOL[dtype]
    assert rel(host(Xg), Xo) <= TOL[dtype]
    assert rows_rel(host(Yg), Yo, B) <= TOL[dtype]
    assert rows_rel(host(Xg), Xo, N) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("case", CASES)
def test_jacobian_parity(ct, case, dtype):
    N, B, vpf, _, offs = case
    theta, delta, X, Y = _case_inputs(N, B, vpf, 1, offs, seed=N * 11 + 1, near_axis=1e-7)
    V = sum(vpf)
    rng = np.random.default_rng(N)
    dth = rng.standard_normal(V)
    ddl = rng.standard_normal(V) if offs else None
    g = oracle.Geometry(N, B, V, vpf)
    op = ct.CTOperator(N, B, V, vpf, max_batch=1, dtype=dtype)
    th, dl = dev(theta), (dev(delta) if delta is not None else None)
    x, r = X[0], Y[0]
    dy = op.jac(dev(x, dtype), th, dev(dth), dl, dev(ddl) if ddl is not None else None)
    gt, gd = op.jacT(dev(x, dtype), th, dev(r, dtype), dl, want_delta=True)
    torch.cuda.synchronize()
    dyo = oracle.jac(g, theta, x, dth, delta, ddl)
    gto, gdo = oracle.jacT(g, theta, x, r, delta)
    assert rel(host(dy), dyo) <= TOL[dtype]
    assert rel(host(gt), gto) <= TOL[dtype]
    assert rel(host(gd), gdo) <= TOL[dtype]
    dt, dd = oracle.dsample(g, theta, x, delta)
    assert rows_rel(host(dy), dyo, B) <= TOL[dtype]
    assert view_sum_rel(host(gt), gto, r, dt, V, B) <= TOL[dtype]
    assert view_sum_rel(host(gd), gdo, r, dd, V, B) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_views_exactly_on_the_diagonals(ct, dtype):
    """Views at the FP64 values of pi/4, 3pi/4 (and those plus pi, minus pi),
    where |cos| and |sin| differ by about one unit in the last place.  The
    axis is decided on theta itself (theta mod pi against the doubles nearest
    pi/4 and 3pi/4, ties to rows), the same on both sides, which matters for J
    and J^T: the Joseph sums are continuous across the diagonal, their angle
    derivative is not.  A detector offset keeps the samples off the
    interpolation kinks that an exact 45 degree view meets, where the one-sided
    slope would depend on the last bit of tan(theta)."""
    N, B = 40, 57
    rng = np.random.default_rng(77)
    theta = np.array([math.pi / 4, 3 * math.pi / 4, math.pi / 4 + math.pi, 3 * math.pi / 4 - math.pi,
                      0.3, 2.0])
    V = theta.size
    g = oracle.Geometry(N, B, V)
    x = rng.uniform(size=N * N)
    r = rng.standard_normal(V * B)
    dth = rng.standard_normal(V)
    delta = np.full(V, 0.1234)
    op = ct.CTOperator(N, B, V, max_batch=1, dtype=dtype)
    th, dl = dev(theta), dev(delta)
    y = op.forward(dev(x, dtype), th, dl)
    xa = op.adjoint(dev(r, dtype), th, dl)
    dy = op.jac(dev(x, dtype), th, dev(dth), dl)
    gt = op.jacT(dev(x, dtype), th, dev(r, dtype), dl)
    torch.cuda.synchronize()
    yo, xo = oracle.forward(g, theta, x, delta), oracle.adjoint(g, theta, r, delta)
    dyo = oracle.jac(g, theta, x, dth, delta)
    gto, _ = oracle.jacT(g, theta, x, r, delta)
    dt, _ = oracle.dsample(g, theta, x, delta)
    assert rows_rel(host(y), yo, B) <= TOL[dtype]
    assert rows_rel(host(xa), xo, N) <= TOL[dtype]
    assert rows_rel(host(dy), dyo, B) <= TOL[dtype]
    assert view_sum_rel(host(gt), gto, r, dt, V, B) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_gauss_newton_terms(ct, dtype):
    N, B, V = 48, 69, 21
    rng = np.random.default_rng(3)
    theta = synth.random_angles(V, rng)
    x = rng.uniform(size=N * N)
    bdata = rng.standard_normal(V * B) * 5
    g = oracle.Geometry(N, B, V)
    op = ct.CTOperator(N, B, V, dtype=dtype, max_batch=1)
    gr, j2, f, res = op.gn_terms(dev(x, dtype), dev(theta), dev(bdata, dtype), want_residual=True)
    torch.cuda.synchronize()
    r_o = oracle.forward(g, theta, x) - bdata
    dt, _ = oracle.dsample(g, theta, x)
    dt = dt.reshape(V, B)
    R = r_o.reshape(V, B)
    assert rel(host(res), r_o) <= TOL[dtype]
    assert rel(host(gr), (R * dt).sum(1)) <= TOL[dtype]
    assert rel(host(j2), (dt * dt).sum(1)) <= TOL[dtype]
    assert rel(host(f), 0.5 * (R * R).sum(1)) <= TOL[dtype]
    assert rows_rel(host(res), r_o, B) <= TOL[dtype]
    assert view_sum_rel(host(gr), (R * dt).sum(1), R, dt, V, B) <= TOL[dtype]
    assert float(np.max(np.abs(host(j2) / (dt * dt).sum(1) - 1))) <= TOL[dtype]
    assert float(np.max(np.abs(host(f) / (0.5 * (R * R).sum(1)) - 1))) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_adjoint_identity_on_gpu(ct, dtype):
    N, B, V = 96, 137, 45
    rng = np.random.default_rng(4)
    theta = synth.random_angles(V, rng)
    op = ct.CTOperator(N, B, V, dtype=dtype, max_batch=1)
    th = dev(theta)
    x = dev(rng.standard_normal(N * N), dtype)
    y = dev(rng.standard_normal(V * B), dtype)
    Ax = op.forward(x, th)
    ATy = op.adjoint(y, th)
    lhs = float((Ax.double() * y.double()).sum())
    rhs = float((x.double() * ATy.double()).sum())
    scale = float(Ax.double().norm() * y.double().norm())
    assert abs(lhs - rhs) / scale <= (1e-6 if dtype == torch.float32 else 1e-14)
    dth = dev(rng.standard_normal(V))
    jd = op.jac(x, th, dth)
    gt = op.jacT(x, th, y)
    lhs = float((jd.double() * y.double()).sum())
    rhs = float((dth * gt).sum())
    assert abs(lhs - rhs) / (float(jd.double().norm() * y.double().norm()) + 1e-300) <= (
        1e-5 if dtype == torch.float32 else 1e-12)


@pytest.fixture(scope="module")
def c2_oracle():
    """The 256^2 / 180-view / 363-bin workload with a batch of 8 and the oracle's
    H, H^T, J and J^T on it (computed once for the launch shapes below)."""
    w = synth.make_workload("C2")
    N, B, V = w.N, w.B, w.V
    g = oracle.Geometry(N, B, V)
    rng = np.random.default_rng(9)
    X = np.concatenate([w.images.reshape(1, -1), rng.uniform(size=(w.batch - 1, N * N))])
    Yo = oracle.forward(g, w.theta_true, X)
    R = rng.standard_normal(Yo.shape)
    Xo = oracle.adjoint(g, w.theta_true, R)
    dth = rng.standard_normal(V)
    dyo = oracle.jac(g, w.theta_true, X[0], dth)
    r = Yo[0] - oracle.forward(g, w.theta_nominal, X[0])
    gto = oracle.jacT(g, w.theta_true, X[0], r)[0]
    dt, _ = oracle.dsample(g, w.theta_true, X[0])
    return dict(w=w, X=X, Yo=Yo, R=R, Xo=Xo, dth=dth, dyo=dyo, r=r, gto=gto, dt=dt)


# the default shapes; the ones the autotuner picks in the benchmark's runs (forward on
# images interleaved in groups of 4, staged transpose in clusters of 4 CTAs); the ones
# it picks here
@pytest.mark.parametrize("shape", ["default", [4, 4, 1, 8, 4, 4, 1, 0, 0, 8, 2, 1], "autotune"])
def test_full_size_workload_parity(ct, c2_oracle, shape):
    """The 256^2 / 180-view / 363-bin workload, batch 8, as the benchmark runs it:
    normwise and per view / per image row against the oracle."""
    o = c2_oracle
    w = o["w"]
    N, B, V = w.N, w.B, w.V
    op = ct.CTOperator(N, B, V, dtype=torch.float32, max_batch=w.batch)
    if shape == "autotune":
        op.autotune()
    elif shape != "default":
        op.tuning = shape
    th = dev(w.theta_true)
    Yg = host(op.forward(dev(o["X"], torch.float32), th))
    assert rel(Yg, o["Yo"]) <= 1e-5 and rows_rel(Yg, o["Yo"], B) <= 1e-5
    Xg = host(op.adjoint(dev(o["R"], torch.float32), th))
    assert rel(Xg, o["Xo"]) <= 1e-5 and rows_rel(Xg, o["Xo"], N) <= 1e-5
    dy = host(op.jac(dev(o["X"][0], torch.float32), th, dev(o["dth"])))
    assert rel(dy, o["dyo"]) <= 1e-5 and rows_rel(dy, o["dyo"], B) <= 1e-5
    gt = host(op.jacT(None, th, dev(o["r"], torch.float32)))  # the image of the J call
    assert rel(gt, o["gto"]) <= 1e-5
    assert view_sum_rel(gt, o["gto"], o["r"], o["dt"], V, B) <= 1e-5
    op.close()


def test_large_image_sampled_views(ct):
    """2048^2 image, 2897 bins: a few views checked against the oracle ray by ray."""
    N = 2048
    B = synth.n_bins(N)
    rng = np.random.default_rng(12)
    V = 4
    theta = synth.random_angles(V, rng)
    ells = synth.random_ellipses(N, 40, rng)
    x = synth.rasterize(N, ells, supersample=2).ravel()
    g = oracle.Geometry(N, B, V)
    op = ct.CTOperator(N, B, V, dtype=torch.float32, max_batch=1)
    th = dev(theta)
    xg = dev(x, torch.float32)
    assert rel(host(op.forward(xg, th)), oracle.forward(g, theta, x)) <= 1e-5
    dth = rng.standard_normal(V)
    assert rel(host(op.jac(xg, th, dev(dth))), oracle.jac(g, theta, x, dth)) <= 1e-5
    y = rng.standard_normal(V * B)
    assert rel(host(op.adjoint(dev(y, torch.float32), th)), oracle.adjoint(g, theta, y)) <= 1e-5


@pytest.mark.parametrize("tuning", [[1, 1, 1, 1, 1, 1, 1, 0, 0, 0, 1, 0], [2, 4, 2, 2, 2, 2, 4, 0, 0, 8, 2, 0],
                                    [8, 8, 2, 8, 4, 8, 2, 0, 0, 16, 4, 0], [4, 2, 8, 1, 4, 4, 4, 0, 4, 0, 1, 0],
                                    [8, 1, 8, 8, 2, 1, 8, 8, 8, 16, 2, 0], [4, 1, 4, 2, 2, 1, 4, 4, 8, 8, 4, 0],
                                    [2, 2, 8, 4, 1, 2, 8, 8, 4, 16, 1, 0], [8, 1, 4, 1, 1, 1, 8, 4, 0, 8, 4, 0],
                                    [4, 4, 1, 8, 2, 4, 1, 0, 0, 8, 2, 1], [8, 2, 8, 4, 4, 2, 2, 0, 0, 0, 4, 1]])
def test_results_do_not_depend_on_launch_shapes(ct, tuning):
    N, B, vpf = 40, 59, [7, 13]
    V = sum(vpf)
    rng = np.random.default_rng(21)
    theta = synth.random_angles(V, rng)
    delta = rng.normal(0, 0.5, V)
    X = rng.uniform(size=(11, 2 * N * N))
    Y = rng.standard_normal((11, V * B))
    dth = rng.standard_normal(V)
    g = oracle.Geometry(N, B, V, vpf)
    op = ct.CTOperator(N, B, V, vpf, max_batch=11, dtype=torch.float32)
    op.tuning = tuning
    assert op.tuning == tuning
    th, dl = dev(theta), dev(delta)
    assert rel(host(op.forward(dev(X, torch.float32), th, dl)), oracle.forward(g, theta, X, delta)) <= 1e-5
    assert rel(host(op.adjoint(dev(Y, torch.float32), th, dl)), oracle.adjoint(g, theta, Y, delta)) <= 1e-5
    assert rel(host(op.jac(dev(X[0], torch.float32), th, dev(dth), dl)),
               oracle.jac(g, theta, X[0], dth, delta)) <= 1e-5
    gt = host(op.jacT(dev(X[0], torch.float32), th, dev(Y[0], torch.float32), dl))
    assert rel(gt, oracle.jacT(g, theta, X[0], Y[0], delta)[0]) <= 1e-5
    # the batched Jacobian products at this shape's images per lane (11 = 4 + 4 + 2 + 1)
    dY = host(op.jac_batch(dev(X, torch.float32), th, dev(dth), dl))
    gb = host(op.jacT_batch(dev(X, torch.float32), th, dev(Y, torch.float32), dl))
    for k in (0, 5, 10):
        assert rel(dY[k], oracle.jac(g, theta, X[k], dth, delta)) <= 1e-5
        assert rel(gb[k], oracle.jacT(g, theta, X[k], Y[k], delta)[0]) <= 1e-5


def test_autotune_picks_valid_shapes(ct):
    w = synth.make_workload("C2")
    op = ct.CTOperator(w.N, w.B, w.V, max_batch=8, dtype=torch.float32)
    t = op.autotune()
    assert len(t) == 12 and all(x in (1, 2, 4, 8) for x in t[:7]) and t[7] in (0, 4, 8) and t[8] in (0, 4, 8)
    assert t[9] in (0, 8, 16) and t[10] in (1, 2, 4) and t[11] in (0, 1)
    assert t[11] == 0 or (t[0] in (4, 8) and t[7] == 0)
    th = dev(w.theta_true)
    x = w.images.reshape(1, -1)
    g = oracle.Geometry(w.N, w.B, w.V)
    assert rel(host(op.forward(dev(x, torch.float32), th)), oracle.forward(g, w.theta_true, x)) <= 1e-5


def test_argument_errors(ct):
    op = ct.CTOperator(16, 23, 4, max_batch=2)
    th = dev(np.zeros(4))
    X = torch.zeros(3, 256, device="cuda")
    Y = torch.zeros(3, 4 * 23, device="cuda")
    with pytest.raises(ct.CTError) as e:
        ct.ct_forward(op.h, th, None, X, Y, 3)  # batch above max_batch
    assert e.value.code == ct.CT_ERR_ARG
    with pytest.raises(ct.CTError):
        ct.ct_forward(op.h, None, None, X, Y, 1)
    bad = dev(np.array([0.1, float("nan"), 0.2, 0.3]))
    op.forward(X[0], bad)
    assert op.status() == ct.CT_ERR_NAN
    assert op.status() == ct.CT_OK  # the flag is cleared once reported
    # the interleaved forward layout: FP32 parallel beam, 4 or 8 images per lane, no staging
    good = [4, 2, 2, 4, 2, 4, 1, 0, 0, 0, 1, 1]
    for bad_t in ([2, 2, 2, 4, 2, 4, 1, 0, 0, 0, 1, 1],   # 2 images per lane
                  [4, 2, 4, 4, 2, 4, 1, 4, 0, 0, 1, 1],   # staged forward
                  good[:11] + [2]):                       # no such layout
        with pytest.raises(ct.CTError) as e:
            op.tuning = bad_t
        assert e.value.code == ct.CT_ERR_ARG
    op.tuning = good
    assert op.tuning == good
    for other in (ct.CTOperator(16, 23, 4, max_batch=2, dtype=torch.float64),
                  ct.CTOperator(16, 23, 4, max_batch=2, dtype=torch.float32, source_distance=40.0)):
        with pytest.raises(ct.CTError) as e:
            other.tuning = good
        assert e.value.code == ct.CT_ERR_ARG
        other.close()


def test_repeat_reruns_the_projection_alone(ct):
    """ct_forward_repeat / ct_adjoint_repeat reproduce the last call bit for bit
    and refuse once another call may have changed the handle's layouts."""
    N, B, V = 48, 68, 25
    rng = np.random.default_rng(31)
    theta = synth.random_angles(V, rng)
    op = ct.CTOperator(N, B, V, max_batch=3, dtype=torch.float32)
    th = dev(theta)
    X = dev(rng.uniform(size=(3, N * N)), torch.float32)
    Y = dev(rng.standard_normal((3, V * B)), torch.float32)
    y0 = op.forward(X, th).clone()
    y1 = torch.zeros_like(y0)
    ct.ct_forward_repeat(op.h, y1, 3)
    assert torch.equal(y0, y1)
    x0 = op.adjoint(Y, th).clone()
    x1 = torch.zeros_like(x0)
    ct.ct_adjoint_repeat(op.h, x1, 2)
    assert torch.equal(x0[:2], x1[:2]) and not x1[2].any()
    for call in (lambda: ct.ct_forward_repeat(op.h, y1, 1),      # an adjoint ran since the forward
                 lambda: ct.ct_adjoint_repeat(op.h, x1, 3 + 1)):  # larger than that call's batch
        with pytest.raises(ct.CTError) as e:
            call()
        assert e.value.code == ct.CT_ERR_ARG
    op.jac(X[0], th, dev(rng.standard_normal(V)))
    with pytest.raises(ct.CTError):
        ct.ct_adjoint_repeat(op.h, x1, 1)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_image_reuse_with_null_x(ct, dtype):
    """x = NULL uses the pair layouts of the previous call that took images, at
    the call's own angles: bit for bit what passing that image again gives; the
    layouts survive calls that take no image and are refused when none is
    current (a fresh handle, after ct_autotune, batch above the laid-out one)."""
    N, B, vpf = 40, 57, [7, 5]
    V = sum(vpf)
    rng = np.random.default_rng(41)
    op = ct.CTOperator(N, B, V, vpf, max_batch=4, dtype=dtype)
    n = op.n
    th1, th2 = dev(synth.random_angles(V, rng)), dev(synth.random_angles(V, rng))
    dl = dev(rng.normal(0, 0.5, V))
    X = dev(rng.uniform(size=(4, n)), dtype)
    R = dev(rng.standard_normal((4, V * B)), dtype)
    dth = dev(rng.standard_normal(V))
    with pytest.raises(ct.CTError) as e:
        op.jac(None, th1, dth)
    assert e.value.code == ct.CT_ERR_ARG

    y_ref = op.forward(X[:3], th2, dl).clone()
    op.forward(X[:3], th1)
    op.adjoint(R, th1)                       # takes no image: the layouts stay
    assert torch.equal(op.forward(None, th2, dl, batch=3), y_ref)   # other angles, same images
    with pytest.raises(ct.CTError):
        op.forward(None, th1, batch=4)       # only 3 images are laid out
    dy_ref = op.jac(X[0], th2, dth, dl).clone()
    g_ref = op.jacT(X[1], th1, R[0], dl, want_delta=True)
    gn_ref = op.gn_terms(X[1], th2, R[1], dl, want_residual=True)
    op.jac(X[0], th1, dth)
    assert torch.equal(op.jac(None, th2, dth, dl), dy_ref)
    op.jacT(X[1], th2, R[3])
    g = op.jacT(None, th1, R[0], dl, want_delta=True)
    assert torch.equal(g[0], g_ref[0]) and torch.equal(g[1], g_ref[1])
    gn = op.gn_terms(None, th2, R[1], dl, want_residual=True)
    assert all(torch.equal(a, b) for a, b in zip(gn, gn_ref))
    # batched forms: the first `batch` images of the last layout
    op.forward(X, th1)
    dY = torch.empty(2, V * B, dtype=dtype, device="cuda")
    ct.ct_jac_batch(op.h, th2, None, None, dth, None, dY, 2)
    assert torch.equal(dY, op.jac_batch(X[:2], th2, dth))
    G = torch.empty(2, V, dtype=torch.float64, device="cuda")
    ct.ct_jacT_batch(op.h, th1, None, None, R[:2], G, None, 2)
    assert torch.equal(G, op.jacT_batch(X[:2], th1, R[:2]))
    # and against the oracle, so a stale layout shared by both forms would show
    g = oracle.Geometry(N, B, V, vpf)
    yo = oracle.forward(g, host(th2), host(X[0]), host(dl))
    assert rel(host(op.forward(None, th2, dl)), yo) <= TOL[dtype]
    op.autotune()
    with pytest.raises(ct.CTError):
        op.jacT(None, th1, R[0])
    op.close()


@pytest.mark.parametrize("kb,split,vw", [(4, 4, 1), (8, 2, 2), (4, 1, 8), (8, 8, 1)])
def test_interleaved_forward_matches_the_pair_form(ct, kb, split, vw):
    """The forward on the interleaved images takes the same taps, fractions and
    sums as on the pair images: the same bits for every batch size (groups of
    8 / 4 and the remainder's 2 and 1), uneven frames with an empty one, and
    offsets; within the FP32 bound of the oracle."""
    N, B, vpf = 37, 55, [9, 0, 6, 4]
    V = sum(vpf)
    rng = np.random.default_rng(61)
    theta = synth.random_angles(V, rng)
    delta = rng.normal(0, 0.7, V)
    F = len(vpf)
    X = rng.uniform(size=(11, F * N * N))
    pairs = ct.CTOperator(N, B, V, vpf, max_batch=11, dtype=torch.float32)
    inter = ct.CTOperator(N, B, V, vpf, max_batch=11, dtype=torch.float32)
    pairs.tuning = [kb, split, vw, 4, 2, 4, 1, 0, 0, 0, 1, 0]
    inter.tuning = [kb, split, vw, 4, 2, 4, 1, 0, 0, 0, 1, 1]
    th, dl = dev(theta), dev(delta)
    Xg = dev(X, torch.float32)
    g = oracle.Geometry(N, B, V, vpf)
    for K in (1, 2, 3, 4, 5, 6, 7, 8, 11):
        y0 = pairs.forward(Xg[:K], th, dl)
        y1 = inter.forward(Xg[:K], th, dl)
        assert torch.equal(y0, y1), K
    yo = oracle.forward(g, theta, X, delta)
    assert rel(host(y1), yo) <= 1e-5
    assert rows_rel(host(y1), yo, B) <= 1e-5
    pairs.close()
    inter.close()


def test_interleaved_layout_reuse(ct):
    """After a forward on interleaved images, x = NULL still means that call's
    images: the forward and its repeat read the interleaved layout again, and
    the Jacobian products (which read pair images) get them converted, bit for
    bit what passing the images gives."""
    N, B, vpf = 33, 47, [6, 5]
    V = sum(vpf)
    rng = np.random.default_rng(62)
    op = ct.CTOperator(N, B, V, vpf, max_batch=7, dtype=torch.float32)
    op.tuning = [4, 2, 2, 4, 2, 4, 1, 0, 0, 0, 2, 1]
    assert op.tuning[11] == 1
    th1, th2 = dev(synth.random_angles(V, rng)), dev(synth.random_angles(V, rng))
    dl = dev(rng.normal(0, 0.5, V))
    X = dev(rng.uniform(size=(7, op.n)), torch.float32)
    R = dev(rng.standard_normal((7, V * B)), torch.float32)
    dth = dev(rng.standard_normal(V))
    y_ref = op.forward(X, th2, dl).clone()
    dY_ref = op.jac_batch(X[:6], th1, dth).clone()
    g_ref = op.jacT(X[0], th2, R[0], dl, want_delta=True)
    g_ref = (g_ref[0].clone(), g_ref[1].clone())
    op.forward(X, th1)
    assert torch.equal(op.forward(None, th2, dl, batch=7), y_ref)
    y1 = torch.zeros_like(y_ref)
    ct.ct_forward_repeat(op.h, y1, 7)
    assert torch.equal(y1, y_ref)
    # batches ending inside a group of the layout (4 + 2 + 1): the images past the
    # batch are read but not written
    for nb in (1, 3, 5, 6):
        y1.zero_()
        ct.ct_forward(op.h, th2, dl, None, y1, nb)
        assert torch.equal(y1[:nb], y_ref[:nb]) and not y1[nb:].any(), nb
        y1.zero_()
        ct.ct_forward_repeat(op.h, y1, nb)
        assert torch.equal(y1[:nb], y_ref[:nb]) and not y1[nb:].any(), nb
    dY = torch.empty(6, V * B, device="cuda")
    ct.ct_jac_batch(op.h, th1, None, None, dth, None, dY, 6)   # converts to pair images
    assert torch.equal(dY, dY_ref)
    g = op.jacT(None, th2, R[0], dl, want_delta=True)
    assert torch.equal(g[0], g_ref[0]) and torch.equal(g[1], g_ref[1])
    # the pair images are current now: the forward reads them and agrees
    assert torch.equal(op.forward(None, th2, dl, batch=7), y_ref)
    op.close()
