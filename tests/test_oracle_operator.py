"""Pins of the FP64 oracle operators against facts that do not come from the oracle itself.

* dense forward matrix == transpose of the dense scatter-adjoint matrix;
* closed forms at theta = 0 and theta = pi/2 (half-pixel column / row sums),
  the detector-offset shift, and the single-pixel hat;
* convergence to the analytic Radon transform of ellipses as N grows;
* convergence of the angle and offset derivatives to the closed-form
  derivatives of the Radon transform of Gaussian blobs (smooth, so the
  derivative converges in norm, unlike that of an ellipse's chord, whose edge
  singularity is not square-integrable);
* central finite differences for d/dtheta and d/ddelta (including the
  global-shift direction of the paper's CT experiments, J * 1);
* closed-form angle / offset derivatives at theta = 0.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_06336_gb300 import synth


def _geom(N, V, B=None):
    return oracle.Geometry(N, B or synth.n_bins(N), V)


def test_dense_forward_equals_transpose_of_scatter_adjoint():
    N, V = 16, 8
    g = _geom(N, V)
    theta = np.array([0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4, 0.3, 1.1, 2.0, 2.9])
    for delta in (None, np.linspace(-0.7, 0.6, V)):
        A = oracle.dense_matrix(g, theta, delta)
        AT = oracle.dense_adjoint_matrix(g, theta, delta)
        assert A.shape == (g.m, g.n)
        assert np.max(np.abs(A - AT.T)) <= 1e-15 * max(1.0, np.max(np.abs(A)))
        assert np.count_nonzero(A) > 0


def test_theta_zero_is_half_pixel_column_sums():
    N = 16
    B = synth.n_bins(N)  # 23, so B - N is odd: bin centres fall between columns
    g = _geom(N, 1, B)
    rng = np.random.default_rng(1)
    X = rng.uniform(size=(N, N))
    Y = oracle.forward(g, np.array([0.0]), X.ravel())
    col = X.sum(axis=0)
    padded = np.concatenate([np.zeros(B), col, np.zeros(B)])
    expect = np.empty(B)
    for b in range(B):
        u = b - (B - 1) / 2 + (N - 1) / 2          # column coordinate of the ray
        j0 = int(math.floor(u))
        expect[b] = 0.5 * (padded[B + j0] + padded[B + j0 + 1])
    np.testing.assert_allclose(Y, expect, rtol=0, atol=1e-13)
    # an offset of half a bin moves the rays onto column centres: plain column sums
    Y2 = oracle.forward(g, np.array([0.0]), X.ravel(), delta=np.array([0.5]))
    u = np.arange(B) - (B - 1) / 2 + 0.5 + (N - 1) / 2
    expect2 = np.array([padded[B + int(round(x))] for x in u])
    np.testing.assert_allclose(Y2, expect2, rtol=0, atol=1e-13)


def test_theta_right_angle_is_half_pixel_row_sums():
    N = 16
    B = synth.n_bins(N)
    g = _geom(N, 1, B)
    rng = np.random.default_rng(2)
    X = rng.uniform(size=(N, N))
    Y = oracle.forward(g, np.array([math.pi / 2]), X.ravel())
    row = X.sum(axis=1)
    padded = np.concatenate([np.zeros(B), row, np.zeros(B)])
    expect = np.empty(B)
    for b in range(B):
        t = (N - 1) / 2 - (b - (B - 1) / 2)         # row coordinate of the ray
        i0 = int(math.floor(t))
        expect[b] = 0.5 * (padded[B + i0] + padded[B + i0 + 1])
    np.testing.assert_allclose(Y, expect, rtol=0, atol=1e-12)


def test_single_pixel_projects_to_a_hat():
    # A unit pixel at (i, j) projects, in view theta, to a triangle centred on
    # xi = x_j cos + y_i sin of half-width a = max(|cos|, |sin|) and height 1/a.
    N = 12
    B = synth.n_bins(N)
    rng = np.random.default_rng(3)
    theta = synth.random_angles(9, rng)
    g = _geom(N, theta.size, B)
    for (i, j) in [(0, 0), (5, 7), (11, 3), (6, 6)]:
        X = np.zeros((N, N))
        X[i, j] = 1.0
        Y = oracle.forward(g, theta, X.ravel()).reshape(theta.size, B)
        x, y = j - (N - 1) / 2, (N - 1) / 2 - i
        for v, th in enumerate(theta):
            c, s = math.cos(th), math.sin(th)
            a = max(abs(c), abs(s))
            xi = x * c + y * s
            sb = np.arange(B) - (B - 1) / 2
            expect = np.maximum(0.0, 1.0 - np.abs(sb - xi) / a) / a
            np.testing.assert_allclose(Y[v], expect, rtol=0, atol=1e-12)


def _radon_ellipses(ells, theta, s):
    """Analytic line integrals of a sum of constant-density ellipses (textbook formula)."""
    out = np.zeros((theta.size, s.size))
    for e in ells:
        for v, th in enumerate(theta):
            t = s - (e.cx * math.cos(th) + e.cy * math.sin(th))
            al2 = (e.a * math.cos(th - e.phi)) ** 2 + (e.b * math.sin(th - e.phi)) ** 2
            inside = t * t < al2
            out[v, inside] += 2.0 * e.rho * e.a * e.b * np.sqrt(al2 - t[inside] ** 2) / al2
    return out


def test_converges_to_analytic_radon_of_ellipses():
    rng = np.random.default_rng(4)
    theta = synth.random_angles(24, rng)
    base = synth.random_ellipses(1, 5, rng)   # unit-size ellipses, scaled with N below
    errs = []
    for N in (32, 64, 128, 256):
        ells = [synth.Ellipse(e.cx * N, e.cy * N, e.a * N, e.b * N, e.phi, e.rho) for e in base]
        X = synth.rasterize(N, ells, supersample=8)
        B = synth.n_bins(N)
        g = _geom(N, theta.size, B)
        Y = oracle.forward(g, theta, X.ravel()).reshape(theta.size, B)
        R = _radon_ellipses(ells, theta, np.arange(B) - (B - 1) / 2)
        errs.append(np.linalg.norm(Y - R) / np.linalg.norm(R))
    # each doubling of the resolution must cut the relative error clearly
    for e0, e1 in zip(errs, errs[1:]):
        assert e1 < 0.8 * e0, errs
    assert errs[-1] < 2e-2, errs


def gaussian_blobs(rng, count=5):
    """Isotropic Gaussians (cx, cy, sigma, rho) in units of the image side, placed so
    that every blob is at least 5 sigma inside the image (truncation below 1e-5)."""
    out = []
    for _ in range(count):
        r, a = 0.2 * math.sqrt(rng.uniform()), rng.uniform(0, 2 * math.pi)
        out.append((r * math.cos(a), r * math.sin(a), rng.uniform(0.03, 0.06), rng.uniform(0.2, 1.0)))
    return out


def gaussian_image(N, blobs):
    """Samples of sum rho exp(-|p - c|^2 / (2 sigma^2)) at the pixel centres."""
    x = np.arange(N) - (N - 1) / 2
    y = (N - 1) / 2 - np.arange(N)
    X = np.zeros((N, N))
    for cx, cy, sg, rho in blobs:
        X += rho * np.exp(-((x[None, :] - cx) ** 2 + (y[:, None] - cy) ** 2) / (2 * sg * sg))
    return X


def _radon_gaussians(blobs, theta, s):
    """Radon transform of the blobs on the lines x cos + y sin = s and its
    derivatives in theta (s fixed) and in s: each blob projects to
    rho sqrt(2 pi) sigma exp(-t^2 / (2 sigma^2)), t = s - c . (cos, sin), and
    dt/dtheta = cx sin - cy cos."""
    c, sn = np.cos(theta)[:, None], np.sin(theta)[:, None]
    R = np.zeros(np.broadcast_shapes(c.shape, s.shape))
    dR_dth, dR_ds = np.zeros_like(R), np.zeros_like(R)
    for cx, cy, sg, rho in blobs:
        t = s - (cx * c + cy * sn)
        gv = rho * math.sqrt(2 * math.pi) * sg * np.exp(-t * t / (2 * sg * sg))
        R += gv
        dR_ds += -t / (sg * sg) * gv
        dR_dth += -t / (sg * sg) * (cx * sn - cy * c) * gv
    return R, dR_dth, dR_ds


def test_derivatives_converge_to_those_of_the_analytic_radon_of_gaussians():
    rng = np.random.default_rng(8)
    V = 24
    theta = synth.random_angles(V, rng)
    delta = rng.normal(0, 0.5, V)
    base = gaussian_blobs(rng)
    errs = []
    for N in (32, 64, 128, 256):
        blobs = [(cx * N, cy * N, sg * N, rho) for (cx, cy, sg, rho) in base]
        X = gaussian_image(N, blobs).ravel()
        B = synth.n_bins(N)
        g = _geom(N, V, B)
        R, R_th, R_s = _radon_gaussians(blobs, theta, np.arange(B) - (B - 1) / 2 + delta[:, None])
        Y = oracle.forward(g, theta, X, delta)
        dt, dd = oracle.dsample(g, theta, X, delta)
        errs.append([np.linalg.norm(a - r.ravel()) / np.linalg.norm(r) for a, r in ((Y, R), (dt, R_th), (dd, R_s))])
    errs = np.array(errs)
    # linear interpolation of a smooth image: O(N^-2) for the projection; the
    # derivatives use the cell slopes, whose O(1/N) errors partly cancel over a ray
    assert np.all(errs[1:, 0] < 0.35 * errs[:-1, 0]), errs
    assert np.all(errs[1:, 1:] < 0.6 * errs[:-1, 1:]), errs
    assert errs[-1, 0] < 1e-3 and np.all(errs[-1, 1:] < 1.5e-2), errs


def _fd_setup(kind, N=32, V=12, seed=5):
    rng = np.random.default_rng(seed)
    theta = synth.random_angles(V, rng, avoid_diagonal=1e-2)
    delta = rng.normal(0, 0.5, V)
    if kind == "phantom":
        X = synth.rasterize(N, synth.random_ellipses(N, 4, rng), supersample=4).ravel()
    else:  # a rough image: every interpolation cell has its own slope
        X = rng.uniform(size=N * N)
    g = _geom(N, V)
    return g, theta, delta, X, rng


@pytest.mark.parametrize("kind", ["phantom", "rough"])
@pytest.mark.parametrize("which", ["theta", "delta", "both", "global_shift"])
def test_jacobian_matches_central_differences(which, kind):
    g, theta, delta, X, rng = _fd_setup(kind)
    V = g.V
    errs = {}
    for h in (1e-3, 1e-4, 1e-5):
        tot_err = tot_ref = 0.0
        for k in range(8):
            if which == "global_shift":
                dth, ddl = np.ones(V), np.zeros(V)
            else:
                dth = rng.standard_normal(V) if which in ("theta", "both") else np.zeros(V)
                ddl = rng.standard_normal(V) if which in ("delta", "both") else np.zeros(V)
            jd = oracle.jac(g, theta, X, dth, delta, ddl)
            fp = oracle.forward(g, theta + h * dth, X, delta + h * ddl)
            fm = oracle.forward(g, theta - h * dth, X, delta - h * ddl)
            fd = (fp - fm) / (2 * h)
            tot_err += np.sum(np.abs(fd - jd))
            tot_ref += np.sum(np.abs(jd))
        errs[h] = tot_err / tot_ref
    # Away from interpolation kinks the central quotient is exact up to O(h^2);
    # kinks crossed inside [-h, h] add an O(h) error in the 1-norm.
    assert errs[1e-4] < 1e-2, errs
    assert errs[1e-5] < max(errs[1e-3] / 30, 1e-9), errs


def test_jacobian_closed_form_at_theta_zero():
    N = 16
    B = synth.n_bins(N)
    g = _geom(N, 1, B)
    rng = np.random.default_rng(6)
    X = rng.uniform(size=(N, N))
    dt, dd = oracle.dsample(g, np.array([0.0]), X.ravel())
    y = (N - 1) / 2 - np.arange(N)
    Xp = np.concatenate([np.zeros((N, B)), X, np.zeros((N, B))], axis=1)
    for b in range(B):
        j0 = int(math.floor(b - (B - 1) / 2 + (N - 1) / 2))
        slope = Xp[:, B + j0 + 1] - Xp[:, B + j0]
        # d/ddelta: column-sum slope; d/dtheta: du/dtheta = -y_i at theta = 0
        assert abs(dd[b] - slope.sum()) < 1e-12
        assert abs(dt[b] - np.sum(slope * (-y))) < 1e-11


def test_adjoint_identity_and_duality():
    rng = np.random.default_rng(7)
    N, V = 24, 17
    g = oracle.Geometry(N, synth.n_bins(N), V, views_per_frame=[9, 8])
    theta = synth.random_angles(V, rng)
    delta = rng.normal(0, 0.5, V)
    x = rng.standard_normal(g.n)
    y = rng.standard_normal(g.m)
    Ax = oracle.forward(g, theta, x, delta)
    ATy = oracle.adjoint(g, theta, y, delta)
    assert abs(Ax @ y - x @ ATy) <= 1e-13 * np.linalg.norm(Ax) * np.linalg.norm(y)
    dth, ddl = rng.standard_normal(V), rng.standard_normal(V)
    gt, gd = oracle.jacT(g, theta, x, y, delta)
    jd = oracle.jac(g, theta, x, dth, delta, ddl)
    assert abs(jd @ y - (dth @ gt + ddl @ gd)) <= 1e-12 * np.linalg.norm(jd) * np.linalg.norm(y)


def test_frames_are_block_diagonal():
    rng = np.random.default_rng(8)
    N = 12
    vpf = [3, 5, 2]
    V = sum(vpf)
    g = oracle.Geometry(N, synth.n_bins(N), V, views_per_frame=vpf)
    theta = synth.random_angles(V, rng)
    x = rng.standard_normal(g.n)
    Y = oracle.forward(g, theta, x)
    start = 0
    for f, nv in enumerate(vpf):
        gf = oracle.Geometry(N, g.B, nv)
        Yf = oracle.forward(gf, theta[start:start + nv], x[f * N * N:(f + 1) * N * N])
        np.testing.assert_array_equal(Y[start * g.B:(start + nv) * g.B], Yf)
        start += nv


def test_joseph_axis_ties_go_to_rows_at_the_fp64_diagonals():
    """The axis rule (rows iff |cos| >= |sin|, decided on theta mod pi against
    the doubles nearest pi/4 and 3pi/4): at those doubles the view is
    row-marched.  The Joseph sums are continuous across the diagonal, their
    angle derivative is not (row- and column-marched interpolation slopes
    differ), so the derivative there equals the one a picoradian inside the
    row-marched side and not the one inside the column-marched side; the same
    one half-turn on and for negative angles."""
    N = 16
    B = synth.n_bins(N)
    rng = np.random.default_rng(5)
    x = rng.uniform(size=N * N)
    q1, q3 = math.pi / 4, 3 * math.pi / 4
    eps = 1e-12
    # (diagonal angle, a row-marched neighbour, a column-marched neighbour)
    cases = [(q1, q1 - eps, q1 + eps), (q3, q3 + eps, q3 - eps), (q1 + math.pi, q1 + math.pi - eps, q1 + math.pi + eps),
             (-q1, -q1 + eps, -q1 - eps), (q3 - math.pi, q3 - math.pi + eps, q3 - math.pi - eps)]
    g = oracle.Geometry(N, B, 1)
    dl = np.array([0.1234])  # moves the samples off the interpolation kinks that an exact 45 degree view meets
    for t, t_rows, t_cols in cases:
        assert abs(math.cos(t_rows)) > abs(math.sin(t_rows)) and abs(math.cos(t_cols)) < abs(math.sin(t_cols))
        y, y_rows, y_cols = (oracle.forward(g, np.array([a]), x, dl) for a in (t, t_rows, t_cols))
        assert np.max(np.abs(y_rows - y_cols)) <= 1e-9 * np.max(np.abs(y))   # H is continuous there
        d, d_rows, d_cols = (oracle.dsample(g, np.array([a]), x, dl)[0] for a in (t, t_rows, t_cols))
        assert np.max(np.abs(d - d_rows)) <= 1e-6 * np.max(np.abs(d)), t
        assert np.max(np.abs(d - d_cols)) > 1e-2 * np.max(np.abs(d)), t
