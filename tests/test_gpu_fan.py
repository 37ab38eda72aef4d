"""GPU parity of the fan-beam operators (handles with source_distance > 0)
against the FP64 fan-beam oracle.

Tolerances as for the parallel beam (normwise relative): float32 1e-5 for H,
H^T, J_theta, J_theta^T and the Gauss-Newton terms; float64 1e-12.  The cases
mix views whose rays all march rows or all march columns with views whose fan
straddles 45 degrees (rays of both kinds in one view), odd image sides, ragged
batches, frames with an empty one, and fixed detector offsets in H and H^T.
Also: the offset derivatives (J_delta, J_delta^T: an offset moves the bin
centres along the detector line), the adjoint identity, the parallel-beam
limit of a distant source, and NL-RMM-GKS on fan-beam data following the
oracle's iterates.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import nlrmm
from paper_2605_06336_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float32: 1e-5, torch.float64: 1e-12}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


CASES = [
    # (N, views_per_frame, batch, D, offsets)
    (16, [10], 3, 20.0, False),
    (37, [11], 11, 60.0, False),          # odd side, batch 8 + 2 + 1
    (24, [4, 1, 0, 6], 2, 40.0, True),    # uneven frames, one empty; fixed offsets
    (64, [90], 8, 128.0, False),
]


def _angles(V, rng):
    # Near the axes (1e-7 off) and fans straddling 45 degrees.  Exactly at
    # theta = 0 a ray of integer s_b has slope s_b / D, and many of its
    # samples fall exactly on an interpolation-cell boundary (s_b y / D a
    # whole or half number); the angle derivative there takes a one-sided
    # slope that the last bit of the sample position decides, which the FP64
    # oracle and the fixed-point kernels round differently (the forward,
    # continuous across the boundary, agrees).
    th = synth.random_angles(V, rng)
    mixed = [1e-7, math.pi / 2 + 1e-7, 0.70, 2.45, math.pi / 4 + 0.05]
    th[:min(V, len(mixed))] = mixed[:min(V, len(mixed))]
    return th


def _inputs(N, vpf, batch, offs, seed):
    rng = np.random.default_rng(seed)
    V = sum(vpf)
    theta = _angles(V, rng)
    delta = rng.normal(0, 0.5, V) if offs else None
    X = rng.uniform(size=(batch, len(vpf) * N * N))
    Y = rng.standard_normal((batch, V * synth.n_bins(N)))
    return theta, delta, X, Y, rng


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{c[0]}_F{len(c[1])}_K{c[2]}")
def test_fan_forward_adjoint_parity(case, dtype):
    from paper_2605_06336_gb300 import ct
    N, vpf, batch, D, offs = case
    B, V = synth.n_bins(N), sum(vpf)
    theta, delta, X, Y, _ = _inputs(N, vpf, batch, offs, seed=N + batch)
    g = oracle.Geometry(N, B, V, vpf, fan_D=D)
    op = ct.CTOperator(N, B, V, vpf, max_batch=batch, dtype=dtype, source_distance=D)
    th, dl = dev(theta), (dev(delta) if delta is not None else None)
    assert rel(host(op.forward(dev(X, dtype), th, dl)), oracle.forward(g, theta, X, delta)) <= TOL[dtype]
    assert rel(host(op.adjoint(dev(Y, dtype), th, dl)), oracle.adjoint(g, theta, Y, delta)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{c[0]}_F{len(c[1])}_K{c[2]}")
def test_fan_jacobian_parity(case, dtype):
    from paper_2605_06336_gb300 import ct
    N, vpf, batch, D, offs = case
    B, V = synth.n_bins(N), sum(vpf)
    theta, delta, X, Y, rng = _inputs(N, vpf, batch, offs, seed=3 * N + batch)
    g = oracle.Geometry(N, B, V, vpf, fan_D=D)
    op = ct.CTOperator(N, B, V, vpf, max_batch=batch, dtype=dtype, source_distance=D)
    th, dl = dev(theta), (dev(delta) if delta is not None else None)
    x, r, dth = X[0], Y[0], rng.standard_normal(V)
    assert rel(host(op.jac(dev(x, dtype), th, dev(dth), dl)), oracle.jac(g, theta, x, dth, delta)) <= TOL[dtype]
    assert rel(host(op.jacT(dev(x, dtype), th, dev(r, dtype), dl)), oracle.jacT(g, theta, x, r, delta)[0]) <= TOL[dtype]
    # fused Gauss-Newton terms: residual, J^T r, |J_v|^2, f_v
    gr, j2, f, res = op.gn_terms(dev(x, dtype), th, dev(r, dtype), dl, want_residual=True)
    r_o = oracle.forward(g, theta, x, delta) - r
    dt = oracle.dsample(g, theta, x, delta)[0].reshape(V, B)
    R = r_o.reshape(V, B)
    assert rel(host(res), r_o) <= TOL[dtype]
    assert rel(host(gr), (R * dt).sum(1)) <= TOL[dtype]
    assert rel(host(j2), (dt * dt).sum(1)) <= TOL[dtype]
    assert rel(host(f), 0.5 * (R * R).sum(1)) <= TOL[dtype]


def test_fan_full_size_256_image_180_views():
    """The 256^2 / 180-view / 363-bin block of the headline workload, fan beam
    with D = 2N, an 8-image batch, in FP32."""
    from paper_2605_06336_gb300 import ct
    w = synth.make_workload("C2")
    D = 2.0 * w.N
    rng = np.random.default_rng(5)
    X = np.concatenate([w.images.reshape(1, -1), rng.uniform(size=(7, w.N * w.N))])
    g = oracle.Geometry(w.N, w.B, w.V, fan_D=D)
    op = ct.CTOperator(w.N, w.B, w.V, max_batch=8, dtype=torch.float32, source_distance=D)
    th = dev(w.theta_true)
    assert rel(host(op.forward(dev(X, torch.float32), th)), oracle.forward(g, w.theta_true, X)) <= 1e-5
    Y = rng.standard_normal((8, w.V * w.B))
    assert rel(host(op.adjoint(dev(Y, torch.float32), th)), oracle.adjoint(g, w.theta_true, Y)) <= 1e-5
    dth = rng.standard_normal(w.V)
    assert rel(host(op.jac(dev(X[0], torch.float32), th, dev(dth))), oracle.jac(g, w.theta_true, X[0], dth)) <= 1e-5
    assert rel(host(op.jacT(dev(X[0], torch.float32), th, dev(Y[0], torch.float32))),
               oracle.jacT(g, w.theta_true, X[0], Y[0])[0]) <= 1e-5


def test_fan_adjoint_identity_and_parallel_limit():
    from paper_2605_06336_gb300 import ct
    N, V = 48, 40
    B = synth.n_bins(N)
    rng = np.random.default_rng(9)
    theta = synth.random_angles(V, rng)
    x, y = rng.standard_normal(N * N), rng.standard_normal(V * B)
    op = ct.CTOperator(N, B, V, max_batch=1, dtype=torch.float64, source_distance=2.0 * N)
    Ax = host(op.forward(dev(x), dev(theta)))
    ATy = host(op.adjoint(dev(y), dev(theta)))
    assert abs(Ax @ y - x @ ATy) <= 1e-13 * np.linalg.norm(Ax) * np.linalg.norm(y)
    far = ct.CTOperator(N, B, V, max_batch=1, dtype=torch.float64, source_distance=1e7)
    par = ct.CTOperator(N, B, V, max_batch=1, dtype=torch.float64)
    yf, yp = host(far.forward(dev(x), dev(theta))), host(par.forward(dev(x), dev(theta)))
    # a distant source: samples move by O(N^2 / D) pixels, which on this rough
    # image changes the projections by ~3e-5 (the oracle gives the same)
    assert rel(yf, yp) <= 1e-4
    assert rel(yf, oracle.forward(oracle.Geometry(N, B, V, fan_D=1e7), theta, x)) <= 1e-12


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("N,vpf,D", [(16, [10], 20.0), (37, [11], 60.0), (24, [4, 1, 0, 6], 40.0),
                                     (64, [90], 128.0)])
def test_fan_offset_derivative_parity(N, vpf, D, dtype):
    """J_theta dtheta + J_delta ddelta and J^T r (both gradients) with per-view
    offsets, against the oracle's fan-beam derivatives (pinned by central
    differences and by Gaussian-blob line integrals); per view as well as
    normwise."""
    from paper_2605_06336_gb300 import ct
    B, V = synth.n_bins(N), sum(vpf)
    theta, _, X, Y, rng = _inputs(N, vpf, 1, False, seed=5 * N + 1)
    delta = rng.normal(0, 0.5, V)
    g = oracle.Geometry(N, B, V, vpf, fan_D=D)
    op = ct.CTOperator(N, B, V, vpf, max_batch=1, dtype=dtype, source_distance=D)
    th, dl = dev(theta), dev(delta)
    x, r = X[0], Y[0]
    dth, ddl = rng.standard_normal(V), rng.standard_normal(V)
    dy = host(op.jac(dev(x, dtype), th, dev(dth), dl, dev(ddl)))
    dyo = oracle.jac(g, theta, x, dth, delta, ddl)
    assert rel(dy, dyo) <= TOL[dtype]
    dyv, dyov = dy.reshape(V, B), dyo.reshape(V, B)
    if V:
        sc = np.maximum(np.abs(dyov).max(1), 1e-300)
        assert float((np.abs(dyv - dyov).max(1) / sc).max()) <= TOL[dtype]
    gt, gd = op.jacT(dev(x, dtype), th, dev(r, dtype), dl, want_delta=True)
    gto, gdo = oracle.jacT(g, theta, x, r, delta)
    assert rel(host(gt), gto) <= TOL[dtype]
    assert rel(host(gd), gdo) <= TOL[dtype]
    dt, dd = oracle.dsample(g, theta, x, delta)
    mag = (np.abs(r.reshape(V, B)) * np.abs(dd.reshape(V, B))).sum(1)
    if V:
        assert float((np.abs(host(gd) - gdo) / np.maximum(mag, 1e-300)).max()) <= TOL[dtype]


def test_fp64_fan_solver_follows_the_oracle_iterates():
    from paper_2605_06336_gb300 import ct
    rng = np.random.default_rng(21)
    N, V = 32, 40
    B, D = synth.n_bins(N), 64.0
    g = oracle.Geometry(N, B, V, fan_D=D)
    th_nom = np.sort(synth.random_angles(V, rng))
    th_true = th_nom + rng.normal(0, math.radians(0.5), V)
    u_true = synth.rasterize(N, synth.random_ellipses(N, 4, rng)).ravel()
    b_true = oracle.forward(g, th_true, u_true)
    e = rng.standard_normal(g.m)
    e *= 0.01 * np.linalg.norm(b_true) / np.linalg.norm(e)
    b, nn = b_true + e, float(np.linalg.norm(e))
    o = nlrmm.Options(noise_norm=nn, k_min=5, k_max=15, outer_iters=4, tol1=0.0, stop_on_convergence=False)
    u_o, th_o, h_o = nlrmm.NLRMMGKS(g, b, o).solve(th_nom, u_true=u_true, theta_true=th_true)
    op = ct.CTOperator(N, B, V, max_batch=8, dtype=torch.float64, source_distance=D)
    x, th, st = op.solve(dev(b), dev(th_nom), x_true=dev(u_true), noise_norm=nn, k_min=5, k_max=15, outer_iters=4,
                         tol1=0.0, stop_on_convergence=0)
    assert st["enlarge_steps"] == h_o.enlarge_steps
    np.testing.assert_allclose(st["lambda"], h_o.lam, rtol=1e-7)
    np.testing.assert_allclose(st["rre"], h_o.rre, rtol=1e-7)
    assert rel(host(x), u_o) <= 1e-7
    assert np.max(np.abs(host(th) - th_o)) <= 1e-8
    assert np.linalg.norm(th_o - th_true) < np.linalg.norm(th_nom - th_true)


def test_fp64_fan_varpro_solver_follows_the_oracle_iterates():
    from paper_2605_06336_gb300 import ct
    rng = np.random.default_rng(23)
    N, V = 32, 40
    B, D = synth.n_bins(N), 64.0
    g = oracle.Geometry(N, B, V, fan_D=D)
    th_nom = np.sort(synth.random_angles(V, rng))
    th_true = th_nom + rng.normal(0, math.radians(0.5), V)
    u_true = synth.rasterize(N, synth.random_ellipses(N, 4, rng)).ravel()
    b_true = oracle.forward(g, th_true, u_true)
    e = rng.standard_normal(g.m)
    e *= 0.01 * np.linalg.norm(b_true) / np.linalg.norm(e)
    b, nn = b_true + e, float(np.linalg.norm(e))
    kw = dict(k_min=5, k_max=15, outer_iters=3, tol1=0.0)
    o = nlrmm.Options(noise_norm=nn, stop_on_convergence=False, varpro=True, **kw)
    u_o, th_o, h_o = nlrmm.NLRMMGKS(g, b, o).solve(th_nom, u_true=u_true)
    op = ct.CTOperator(N, B, V, max_batch=8, dtype=torch.float64, source_distance=D)
    x, th, st = op.solve(dev(b), dev(th_nom), x_true=dev(u_true), noise_norm=nn, stop_on_convergence=0, varpro=1,
                         **kw)
    assert st["enlarge_steps"] == h_o.enlarge_steps
    np.testing.assert_allclose(st["lambda"], h_o.lam, rtol=1e-6)
    np.testing.assert_allclose(st["rre"], h_o.rre, rtol=1e-6)
    assert rel(host(x), u_o) <= 1e-6
    assert np.max(np.abs(host(th) - th_o)) <= 1e-7


def test_fan_image_reuse_with_null_x():
    """Fan beam, x = NULL: the J^T (and J, and H) of the image laid out by the
    previous call, at other angles, bit for bit what passing the image gives."""
    from paper_2605_06336_gb300 import ct
    N, vpf, K, D = 37, [11], 3, 60.0
    theta, delta, X, Y, rng = _inputs(N, vpf, K, True, seed=71)
    V = sum(vpf)
    op = ct.CTOperator(N, synth.n_bins(N), V, max_batch=K, dtype=torch.float32, source_distance=D)
    th1, th2, dl = dev(theta), dev(_angles(V, rng)), dev(delta)
    Xd, Yd = dev(X, torch.float32), dev(Y, torch.float32)
    dth = dev(rng.standard_normal(V))
    g_ref = op.jacT(Xd[1], th2, Yd[0], dl, want_delta=True)
    dy_ref = op.jac(Xd[1], th1, dth, dl).clone()
    y_ref = op.forward(Xd[:2], th2, dl).clone()
    op.forward(Xd, th1)
    op.jac(Xd[1], th2, dth)
    g = op.jacT(None, th2, Yd[0], dl, want_delta=True)
    assert torch.equal(g[0], g_ref[0]) and torch.equal(g[1], g_ref[1])
    assert torch.equal(op.jac(None, th1, dth, dl), dy_ref)
    op.forward(Xd, th1)
    assert torch.equal(op.forward(None, th2, dl, batch=2), y_ref)
    op.close()
