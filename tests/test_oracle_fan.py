"""Pins of the FP64 fan-beam oracle against facts that do not come from the oracle itself.

Fan-beam reading: point source at distance D from the rotation centre, flat
detector rescaled to the line through the centre (the parallel-beam bin
centres s_b on it); ray (v, b) runs from the source through s_b e(theta_v).

* dense fan forward matrix == transpose of the dense scatter-adjoint matrix,
  with views whose rays switch between row and column marching;
* as D grows the fan operator and its derivatives tend to the parallel-beam
  ones (the limit the reading is built on);
* convergence to the analytic line integrals of ellipses along the fan rays;
* convergence of the angle and offset derivatives to the derivatives of the
  closed-form line integrals of Gaussian blobs along the fan rays;
* central finite differences for d/dtheta and d/ddelta;
* adjoint identity and J / J^T duality with frames and offsets.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_06336_gb300 import synth


def _fan(N, V, D, vpf=None):
    return oracle.Geometry(N, synth.n_bins(N), V, vpf, fan_D=D)


def _mixed_angles(V):
    # 45 degrees +- a few: the fan's edge rays then march rows while its other rays march columns
    base = np.array([0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4, 0.3, 1.1, 2.0, 2.9, 0.70, 2.45])
    return base[:V]


def test_fan_dense_forward_equals_transpose_of_scatter_adjoint():
    N, V = 16, 10
    g = _fan(N, V, D=20.0)
    theta = _mixed_angles(V)
    for delta in (None, np.linspace(-0.7, 0.6, V)):
        A = oracle.dense_matrix(g, theta, delta)
        AT = oracle.dense_adjoint_matrix(g, theta, delta)
        assert np.max(np.abs(A - AT.T)) <= 1e-15 * max(1.0, np.max(np.abs(A)))
        assert np.count_nonzero(A) > 0
    # some view really mixes row- and column-marched rays: at 0.70 rad the
    # directions of the fan straddle 45 degrees
    s = np.arange(g.B) - (g.B - 1) / 2
    c, sn = math.cos(0.70), math.sin(0.70)
    rows = np.abs(s * c - 20.0 * sn) <= np.abs(s * sn + 20.0 * c)
    assert rows.any() and (~rows).any()


def test_fan_tends_to_parallel_beam_as_the_source_recedes():
    rng = np.random.default_rng(11)
    N, V = 32, 12
    theta = synth.random_angles(V, rng, avoid_diagonal=1e-2)
    delta = rng.normal(0, 0.5, V)
    X = synth.rasterize(N, synth.random_ellipses(N, 4, rng), supersample=4).ravel()
    gp = oracle.Geometry(N, synth.n_bins(N), V)
    yp = oracle.forward(gp, theta, X, delta)
    dtp, ddp = oracle.dsample(gp, theta, X, delta)
    errs = []
    for D in (1e3, 1e5, 1e7):
        gf = _fan(N, V, D)
        errs.append(np.linalg.norm(oracle.forward(gf, theta, X, delta) - yp) / np.linalg.norm(yp))
    # a fan ray tilts by O(s_b / D) against its parallel ray, so the sample
    # positions move by O(N^2 / D) pixels: the difference falls like 1 / D
    assert errs[1] < errs[0] / 30 and errs[2] < errs[1] / 30, errs
    assert errs[2] < 1e-5, errs
    dtf, ddf = oracle.dsample(_fan(N, V, 1e7), theta, X, delta)
    assert np.linalg.norm(dtf - dtp) <= 1e-5 * np.linalg.norm(dtp)
    assert np.linalg.norm(ddf - ddp) <= 1e-5 * np.linalg.norm(ddp)


def _line_integrals_of_ellipses(ells, phi, p):
    """Analytic integrals of constant-density ellipses along the lines
    { X : X . (cos phi, sin phi) = p } (textbook chord formula)."""
    out = np.zeros(phi.shape)
    for e in ells:
        t = p - (e.cx * np.cos(phi) + e.cy * np.sin(phi))
        al2 = (e.a * np.cos(phi - e.phi)) ** 2 + (e.b * np.sin(phi - e.phi)) ** 2
        inside = t * t < al2
        out[inside] += 2.0 * e.rho * e.a * e.b * np.sqrt(al2[inside] - t[inside] ** 2) / al2[inside]
    return out


def test_fan_converges_to_analytic_line_integrals_of_ellipses():
    rng = np.random.default_rng(4)
    theta = synth.random_angles(24, rng)
    base = synth.random_ellipses(1, 5, rng)
    errs = []
    for N in (32, 64, 128, 256):
        D = 2.0 * N
        ells = [synth.Ellipse(e.cx * N, e.cy * N, e.a * N, e.b * N, e.phi, e.rho) for e in base]
        X = synth.rasterize(N, ells, supersample=8)
        B = synth.n_bins(N)
        g = oracle.Geometry(N, B, theta.size, fan_D=D)
        Y = oracle.forward(g, theta, X.ravel()).reshape(theta.size, B)
        # ray (v, b): through S = D (sin, -cos) and P_b = s_b (cos, sin); unit normal n, offset n . P_b
        s = np.arange(B) - (B - 1) / 2
        c, sn = np.cos(theta)[:, None], np.sin(theta)[:, None]
        rx, ry = s * c - D * sn, s * sn + D * c
        phi = np.arctan2(-rx, ry)
        p = np.cos(phi) * s * c + np.sin(phi) * s * sn
        R = _line_integrals_of_ellipses(ells, phi, p)
        errs.append(np.linalg.norm(Y - R) / np.linalg.norm(R))
    for e0, e1 in zip(errs, errs[1:]):
        assert e1 < 0.8 * e0, errs
    assert errs[-1] < 2e-2, errs


def _fan_gaussian_integrals(blobs, theta, delta, B, D):
    """Closed-form integrals of isotropic Gaussians along the fan rays: a blob
    contributes rho sqrt(2 pi) sigma exp(-t^2 / (2 sigma^2)), t its signed
    distance from the ray through S = D (sin, -cos) and P_b = s_b (cos, sin)."""
    s = np.arange(B) - (B - 1) / 2 + delta[:, None]
    c, sn = np.cos(theta)[:, None], np.sin(theta)[:, None]
    rx, ry = s * c - D * sn, s * sn + D * c
    nr = np.hypot(rx, ry)
    nx, ny = ry / nr, -rx / nr
    p = nx * s * c + ny * s * sn
    R = np.zeros(s.shape)
    for cx, cy, sg, rho in blobs:
        t = p - (nx * cx + ny * cy)
        R += rho * math.sqrt(2 * math.pi) * sg * np.exp(-t * t / (2 * sg * sg))
    return R


def test_fan_derivatives_converge_to_those_of_gaussian_line_integrals():
    rng = np.random.default_rng(8)
    V = 24
    theta = synth.random_angles(V, rng)
    delta = rng.normal(0, 0.5, V)
    base = []
    for _ in range(5):   # blobs at least 5 sigma inside the image
        r, a = 0.2 * math.sqrt(rng.uniform()), rng.uniform(0, 2 * math.pi)
        base.append((r * math.cos(a), r * math.sin(a), rng.uniform(0.03, 0.06), rng.uniform(0.2, 1.0)))
    errs = []
    for N in (32, 64, 128, 256):
        D = 2.0 * N
        blobs = [(cx * N, cy * N, sg * N, rho) for (cx, cy, sg, rho) in base]
        x = np.arange(N) - (N - 1) / 2
        y = (N - 1) / 2 - np.arange(N)
        X = sum(rho * np.exp(-((x[None, :] - cx) ** 2 + (y[:, None] - cy) ** 2) / (2 * sg * sg))
                for cx, cy, sg, rho in blobs).ravel()
        B = synth.n_bins(N)
        g = oracle.Geometry(N, B, V, fan_D=D)
        R = _fan_gaussian_integrals(blobs, theta, delta, B, D)
        # derivatives of the closed form by central differences of the closed
        # form itself (smooth: error ~1e-10, far below the discretization error)
        h = 1e-6
        R_th = (_fan_gaussian_integrals(blobs, theta + h, delta, B, D)
                - _fan_gaussian_integrals(blobs, theta - h, delta, B, D)) / (2 * h)
        R_s = (_fan_gaussian_integrals(blobs, theta, delta + h, B, D)
               - _fan_gaussian_integrals(blobs, theta, delta - h, B, D)) / (2 * h)
        Y = oracle.forward(g, theta, X, delta)
        dt, dd = oracle.dsample(g, theta, X, delta)
        errs.append([np.linalg.norm(a - r.ravel()) / np.linalg.norm(r) for a, r in ((Y, R), (dt, R_th), (dd, R_s))])
    errs = np.array(errs)
    assert np.all(errs[1:, 0] < 0.35 * errs[:-1, 0]), errs
    assert np.all(errs[1:, 1:] < 0.6 * errs[:-1, 1:]), errs
    assert errs[-1, 0] < 1e-3 and np.all(errs[-1, 1:] < 1.5e-2), errs


@pytest.mark.parametrize("which", ["theta", "delta", "both"])
def test_fan_jacobian_matches_central_differences(which):
    rng = np.random.default_rng(5)
    N, V = 32, 12
    g = _fan(N, V, D=64.0)
    theta = synth.random_angles(V, rng, avoid_diagonal=1e-2)
    delta = rng.normal(0, 0.5, V)
    X = synth.rasterize(N, synth.random_ellipses(N, 4, rng), supersample=4).ravel()
    errs = {}
    for h in (1e-3, 1e-4, 1e-5):
        tot_err = tot_ref = 0.0
        for _ in range(8):
            dth = rng.standard_normal(V) if which in ("theta", "both") else np.zeros(V)
            ddl = rng.standard_normal(V) if which in ("delta", "both") else np.zeros(V)
            jd = oracle.jac(g, theta, X, dth, delta, ddl)
            fd = (oracle.forward(g, theta + h * dth, X, delta + h * ddl)
                  - oracle.forward(g, theta - h * dth, X, delta - h * ddl)) / (2 * h)
            tot_err += np.sum(np.abs(fd - jd))
            tot_ref += np.sum(np.abs(jd))
        errs[h] = tot_err / tot_ref
    assert errs[1e-4] < 1e-2, errs
    assert errs[1e-5] < max(errs[1e-3] / 30, 1e-9), errs


def test_fan_adjoint_identity_and_duality():
    rng = np.random.default_rng(7)
    N, V = 24, 17
    g = _fan(N, V, D=40.0, vpf=[9, 8])
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
