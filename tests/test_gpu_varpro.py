"""VarPro on the GPU (nlrmm_varpro, nlrmm_varpro_update, autograd, the
solver's VarPro update) against the oracle.

f(theta) = min_y 1/2 |H(theta) V y - b|^2 + lam/2 |P Psi V y|^2 on a fixed basis V
with frozen MM weights; grad f = J_theta(V y)^T (H V y - b).  The autograd
Function recomputes the reduced solve in backward (nothing stored).
The Gauss-Newton update (Alg. "UPDATE-PARAM-VarPro") solves the damped
system of the sensitivity-equation Jacobians by the Woodbury identity; the
oracle forms them column by column and solves densely.
* one update (1 and 3 Gauss-Newton steps) on 64^2 / 45 views with offsets:
  FP64 angles within 1e-9 rad of the oracle's and the objective history
  within 1e-9 (relative); FP32 operators: the angle change within 1e-3
  (relative) of the oracle's;
* zero-residual problem: quadratic convergence to the true angles (FP64);
* NL-RMM-GKS with the VarPro update: FP64 follows the oracle's iterates,
  FP32 reaches the oracle's reconstruction error within 1e-3 (relative);
* argument errors.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import nlrmm
from paper_2605_06336_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem():
    w = synth.make_workload("C3", scale=0.125)   # 64^2, 45 views, offsets
    g = oracle.Geometry(w.N, w.B, w.V)
    u_true = w.images.reshape(-1)
    b_true = oracle.forward(g, w.theta_true, u_true, w.delta_true)
    e = w.noise_dir * (w.noise_level * np.linalg.norm(b_true) / np.linalg.norm(w.noise_dir))
    b = b_true + e
    s = nlrmm.NLRMMGKS(g, b, nlrmm.Options(noise_norm=float(np.linalg.norm(e))), delta=w.delta_true)
    V = s.gkb(w.theta_nominal, 8)
    u_w = V @ np.linspace(1.0, 0.2, 8)
    return w, g, b, V, u_w


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-9), (torch.float32, 2e-4)])
def test_varpro_value_and_gradient_match_the_oracle(dtype, tol):
    from paper_2605_06336_gb300 import ct
    w, g, b, V, u_w = _problem()
    lam, eps = 0.3, 1e-2
    wts = nlrmm.mm_weights(nlrmm.psi(g, u_w), eps)
    gt_o, f_o, u_o = nlrmm.varpro_gradient(g, b, w.theta_nominal, V, lam, wts, w.delta_true)
    op = ct.CTOperator(w.N, w.B, w.V, max_batch=4, dtype=dtype)
    dv = lambda a, t=dtype: torch.tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    f, grad, u = op.varpro(dv(b), dv(w.theta_nominal, torch.float64), dv(V.T), lam, dv(u_w), eps,
                           delta=dv(w.delta_true, torch.float64))
    assert abs(float(f) - f_o) <= tol * abs(f_o)
    rel = lambda a, c: np.linalg.norm(a - c) / np.linalg.norm(c)
    assert rel(u.double().cpu().numpy(), u_o) <= tol
    # the gradient sums residual x derivative over bins with little cancellation
    # (sum |r||J| / |sum r J| is about 1.4 here), and rounding V, b and the
    # weights to float32 moves the oracle's gradient by 3e-7: no looser bound
    # than for f and u is justified
    assert rel(grad.cpu().numpy(), gt_o) <= tol


def test_autograd_varpro_recomputes_and_matches():
    from paper_2605_06336_gb300 import ct
    from paper_2605_06336_gb300.autograd import varpro_objective
    w, g, b, V, u_w = _problem()
    op = ct.CTOperator(w.N, w.B, w.V, max_batch=4, dtype=torch.float64)
    dv = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    th = dv(w.theta_nominal).requires_grad_(True)
    f = varpro_objective(th, op, dv(b), dv(V.T), 0.3)
    f.backward()
    gt_o, f_o, _ = nlrmm.varpro_gradient(g, b, w.theta_nominal, V, 0.3, None)
    assert abs(float(f.detach()) - f_o) <= 1e-9 * abs(f_o)
    assert np.linalg.norm(th.grad.cpu().numpy() - gt_o) <= 1e-8 * np.linalg.norm(gt_o)


def _rel(a, c):
    return np.linalg.norm(a - c) / np.linalg.norm(c)


@pytest.mark.parametrize("steps", [1, 3])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_varpro_update_matches_the_oracle(dtype, steps):
    from paper_2605_06336_gb300 import ct
    w, g, b, V, u_w = _problem()
    lam, eps = 0.3, 1e-2
    wts = nlrmm.mm_weights(nlrmm.psi(g, u_w), eps)
    unit = 2.0 ** -53 if dtype == torch.float64 else 2.0 ** -24   # Armijo noise floor of the misfit's precision
    s = nlrmm.NLRMMGKS(g, b, nlrmm.Options(maxiter_p=steps, armijo_eps=unit), delta=w.delta_true)
    th_o = s.update_param_varpro(w.theta_nominal, V, lam, wts)
    op = ct.CTOperator(w.N, w.B, w.V, max_batch=4, dtype=dtype)
    dv = lambda a, t=dtype: torch.tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    th, f_hist = op.varpro_update(dv(b), dv(w.theta_nominal, torch.float64), dv(V.T), lam, dv(u_w), eps,
                                  delta=dv(w.delta_true, torch.float64), maxiter_p=steps)
    th = th.cpu().numpy()
    step_o = th_o - w.theta_nominal
    assert np.linalg.norm(step_o) > 1e-3  # the update moves the angles
    if dtype == torch.float64:
        assert np.max(np.abs(th - th_o)) <= 1e-9, np.max(np.abs(th - th_o))
        f_o = [nlrmm.varpro_objective(g, b, w.theta_nominal, V, lam, wts, w.delta_true)[0]]
        t = w.theta_nominal.copy()
        for _ in range(steps):
            t = nlrmm.NLRMMGKS(g, b, nlrmm.Options(maxiter_p=1), delta=w.delta_true).update_param_varpro(
                t, V, lam, wts)
            f_o.append(nlrmm.varpro_objective(g, b, t, V, lam, wts, w.delta_true)[0])
        np.testing.assert_allclose(f_hist, f_o, rtol=1e-9)
    else:
        assert _rel(th - w.theta_nominal, step_o) <= 1e-3, _rel(th - w.theta_nominal, step_o)
    assert all(f_hist[i + 1] <= f_hist[i] for i in range(steps))


def test_varpro_update_converges_quadratically_on_zero_residual_data():
    from paper_2605_06336_gb300 import ct
    N, Vn, k = 32, 24, 6
    rng = np.random.default_rng(15)
    B = synth.n_bins(N)
    g = oracle.Geometry(N, B, Vn)
    th_true = np.sort(synth.random_angles(Vn, rng))
    u_true = synth.rasterize(N, synth.random_ellipses(N, 4, rng)).ravel()
    b = oracle.forward(g, th_true, u_true)
    Vb, _ = np.linalg.qr(np.column_stack([u_true, rng.standard_normal((g.n, k - 1))]))
    th0 = th_true + rng.normal(0, math.radians(0.5), Vn)
    op = ct.CTOperator(N, B, Vn, max_batch=4, dtype=torch.float64)
    dv = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    th = dv(th0)
    errs = []
    for _ in range(4):
        th, _ = op.varpro_update(dv(b), th, dv(Vb.T), 1e-10, maxiter_p=1)
        errs.append(float(np.max(np.abs(th.cpu().numpy() - th_true))))
    assert errs[2] <= 1e-9, errs


def _solver_problem(N, V, seed, noise=0.01, sigma_deg=0.5):
    rng = np.random.default_rng(seed)
    g = oracle.Geometry(N, synth.n_bins(N), V)
    th_nom = np.sort(synth.random_angles(V, rng))
    th_true = th_nom + rng.normal(0, math.radians(sigma_deg), V)
    u_true = synth.rasterize(N, synth.random_ellipses(N, 4, rng)).ravel()
    b_true = oracle.forward(g, th_true, u_true)
    e = rng.standard_normal(g.m)
    e *= noise * np.linalg.norm(b_true) / np.linalg.norm(e)
    return g, th_nom, th_true, u_true, b_true + e, float(np.linalg.norm(e))


def test_fp64_varpro_solver_follows_the_oracle_iterates():
    from paper_2605_06336_gb300 import ct
    g, th_nom, th_true, u_true, b, nn = _solver_problem(32, 40, seed=1)
    o = nlrmm.Options(noise_norm=nn, k_min=5, k_max=15, outer_iters=4, tol1=0.0, stop_on_convergence=False,
                      varpro=True)
    u_o, th_o, h_o = nlrmm.NLRMMGKS(g, b, o).solve(th_nom, u_true=u_true, theta_true=th_true)
    op = ct.CTOperator(g.N, g.B, g.V, max_batch=8, dtype=torch.float64)
    dv = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    x, th, st = op.solve(dv(b), dv(th_nom), x_true=dv(u_true), noise_norm=nn, k_min=5, k_max=15, outer_iters=4,
                         tol1=0.0, stop_on_convergence=0, varpro=1)
    assert st["enlarge_steps"] == h_o.enlarge_steps
    # Gauss-Newton quotients amplify the rounding differences of the two FP64 paths
    np.testing.assert_allclose(st["lambda"], h_o.lam, rtol=1e-6)
    np.testing.assert_allclose(st["rre"], h_o.rre, rtol=1e-6)
    assert _rel(x.cpu().numpy(), u_o) <= 1e-6
    assert np.max(np.abs(th.cpu().numpy() - th_o)) <= 1e-7
    assert np.linalg.norm(th_o - th_true) < 0.7 * np.linalg.norm(th_nom - th_true)


def test_fp32_varpro_solver_reaches_the_oracle_reconstruction_error():
    from paper_2605_06336_gb300 import ct
    w = synth.make_workload("C1")
    g = oracle.Geometry(w.N, w.B, w.V)
    u_true = w.images.reshape(-1)
    b_true = oracle.forward(g, w.theta_true, u_true)
    e = w.noise_dir * (w.noise_level * np.linalg.norm(b_true) / np.linalg.norm(w.noise_dir))
    b = b_true + e
    nn = float(np.linalg.norm(e))
    iters = min(w.outer_iters, 6)
    o = nlrmm.Options(noise_norm=nn, outer_iters=iters, stop_on_convergence=False, varpro=True,
                      armijo_eps=2.0 ** -24)
    u_o, th_o, h_o = nlrmm.NLRMMGKS(g, b, o).solve(w.theta_nominal, u_true=u_true, theta_true=w.theta_true)
    op = ct.CTOperator(w.N, w.B, w.V, max_batch=8, dtype=torch.float32)
    dv = lambda a, t=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    x, th, st = op.solve(dv(b, torch.float32), dv(w.theta_nominal), x_true=dv(u_true, torch.float32),
                         noise_norm=nn, outer_iters=iters, stop_on_convergence=0, varpro=1)
    assert abs(st["rre"][-1] - h_o.rre[-1]) <= 1e-3 * h_o.rre[-1], (st["rre"][-1], h_o.rre[-1])
    ang_gpu = np.linalg.norm(th.cpu().numpy() - w.theta_true) / np.linalg.norm(w.theta_true)
    assert ang_gpu <= 1.05 * h_o.angle_err[-1], (ang_gpu, h_o.angle_err[-1])


def test_varpro_update_argument_errors():
    from paper_2605_06336_gb300 import ct
    op = ct.CTOperator(16, 23, 6, max_batch=2, dtype=torch.float64)
    b = torch.zeros(6 * 23, dtype=torch.float64, device="cuda")
    th = torch.zeros(6, dtype=torch.float64, device="cuda")
    for V, lam in ((torch.zeros(33, 256, dtype=torch.float64, device="cuda"), 1.0),
                   (torch.zeros(4, 256, dtype=torch.float64, device="cuda"), 0.0)):
        with pytest.raises(ct.CTError) as e:
            op.varpro_update(b, th, V, lam)
        assert e.value.code == ct.CT_ERR_ARG


def _moving(N=24, vpf=(6, 7, 6, 7), seed=51):
    rng = np.random.default_rng(seed)
    ells = synth.random_ellipses(N, 3, rng)
    u_true = np.stack([synth.rasterize(N, ells, shift=(0.5 * f, 0.0)) for f in range(len(vpf))]).ravel()
    g = oracle.Geometry(N, synth.n_bins(N), sum(vpf), views_per_frame=list(vpf))
    th_nom = np.sort(synth.random_angles(g.V, rng))
    th_true = th_nom + rng.normal(0, math.radians(0.5), g.V)
    b_true = oracle.forward(g, th_true, u_true)
    e = rng.standard_normal(g.m)
    e *= 0.01 * np.linalg.norm(b_true) / np.linalg.norm(e)
    return g, list(vpf), th_nom, u_true, b_true + e, float(np.linalg.norm(e))


def _follows(st, h_o, x, u_o, th, th_o):
    # Gauss-Newton quotients amplify the rounding differences of the two FP64 paths
    assert st["enlarge_steps"] == h_o.enlarge_steps
    np.testing.assert_allclose(st["lambda"], h_o.lam, rtol=1e-6)
    np.testing.assert_allclose(st["rre"], h_o.rre, rtol=1e-6)
    assert _rel(x, u_o) <= 1e-6
    assert np.max(np.abs(th - th_o)) <= 1e-7


def test_fp64_varpro_with_aniso_tv_follows_the_oracle_iterates():
    from paper_2605_06336_gb300 import ct
    g, vpf, th_nom, u_true, b, nn = _moving()
    kw = dict(k_min=5, k_max=15, outer_iters=3, tol1=0.0)
    o = nlrmm.Options(noise_norm=nn, stop_on_convergence=False, temporal=True, varpro=True, **kw)
    u_o, th_o, h_o = nlrmm.NLRMMGKS(g, b, o).solve(th_nom, u_true=u_true)
    op = ct.CTOperator(g.N, g.B, g.V, vpf, max_batch=8, dtype=torch.float64)
    dv = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    x, th, st = op.solve(dv(b), dv(th_nom), x_true=dv(u_true), noise_norm=nn, stop_on_convergence=0, temporal=1,
                         varpro=1, **kw)
    _follows(st, h_o, x.cpu().numpy(), u_o, th.cpu().numpy(), th_o)


def test_fp64_varpro_streaming_follows_the_oracle_iterates():
    from paper_2605_06336_gb300 import ct
    rng = np.random.default_rng(52)
    N, V, nblocks = 32, 36, 3
    B = synth.n_bins(N)
    g = oracle.Geometry(N, B, V)
    th_nom = np.sort(synth.random_angles(V, rng))
    th_true = th_nom + rng.normal(0, math.radians(0.5), V)
    u_true = synth.rasterize(N, synth.random_ellipses(N, 4, rng)).ravel()
    b_true = oracle.forward(g, th_true, u_true).reshape(V, B)
    e = rng.standard_normal(b_true.shape)
    e *= 0.01 * np.linalg.norm(b_true) / np.linalg.norm(e)
    idx = [np.sort(ix) for ix in np.array_split(rng.permutation(V), nblocks)]
    kw = dict(k_min=5, k_max=15, tol1=0.0)
    orc = [nlrmm.NLRMMGKS(oracle.Geometry(N, B, len(ix)), (b_true[ix] + e[ix]).ravel(),
                          nlrmm.Options(noise_norm=float(np.linalg.norm(e[ix])), stop_on_convergence=False,
                                        varpro=True, **kw)) for ix in idx]
    u_o, th_o, h_o = nlrmm.stream_solve(orc, [th_nom[ix] for ix in idx], passes=2, u_true=u_true)
    dv = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    ops = [ct.CTOperator(N, B, len(ix), max_batch=8, dtype=torch.float64) for ix in idx]
    x, th, st = ct.stream_solve(ops, [dv((b_true[ix] + e[ix]).ravel()) for ix in idx], [dv(th_nom[ix]) for ix in idx],
                                [float(np.linalg.norm(e[ix])) for ix in idx], x_true=dv(u_true), outer_iters=2,
                                stop_on_convergence=0, varpro=1, **kw)
    _follows(st, h_o, x.cpu().numpy(), u_o, np.concatenate([t.cpu().numpy() for t in th]), np.concatenate(th_o))
