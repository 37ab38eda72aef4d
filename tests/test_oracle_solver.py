"""Pins of the FP64 NL-RMM-GKS oracle against mathematics it must satisfy.

* Psi is the stacked Kronecker finite-difference operator and Psi^T its transpose;
* the MM majorant touches J at u_k and lies above it (properties (i), (iii), Sec. 3.1);
* the orthogonalization of new basis vectors (two classical Gram-Schmidt passes) leaves
  a vector orthogonal to V to rounding even when it lies almost in span(V), where one
  pass fails;
* the Golub-Kahan start basis spans the Krylov space K_k(H^T H, H^T b), starts along
  H^T b, is orthonormal, and V^T H^T H V is tridiagonal (the Lanczos relation);
* with fixed lambda and fixed weights the generalized Krylov iteration reaches
  the dense normal-equation solution once V spans the image space;
* fixed-lambda Enlarge steps never increase J_{eps,lambda} (Lemma on image descent);
* with the angles held (Alg. "NL-RMM-GKS" reduced to Alg. "RMM-GKS"), fixed lambda and
  fixed weights, the restarted outer loop (Enlarge, Compress, residual append) never
  increases J and converges to the dense normal-equation solution, even with a basis
  far smaller than the image space; the same holds for the dynamic form, whose Psi
  adds the frame-to-frame differences (ANISO-TV), on frames with uneven view counts;
* after Compress u lies in span(V) and V has orthonormal columns; the retained
  directions are the dominant eigenvectors of V^T (H^T H + lambda Psi^T P^2 Psi) V formed
  from the dense matrices (the leading right singular vectors of [R_H; sqrt(lambda) R_Psi]);
* the discrepancy-principle lambda hits the target residual; targets out of reach give
  the ends of the bracket, and the projected residual increases with lambda;
* the per-view Gauss-Newton / Armijo update reaches the brute-force minimizer of a
  single view's misfit;
* a small alternating solve reduces both the image and the angle error;
* VarPro (Sec. 4.2): the sensitivity-equation Jacobians of the reduced
  residuals r(theta), s(theta) match central differences of those residuals;
  J_r^T r + lambda J_s^T s equals the envelope gradient; on a zero-residual
  problem the Gauss-Newton / Armijo update decreases the reduced objective at
  every step and converges quadratically to the true angles; a small VarPro
  solve reduces both errors;
* streaming (Alg. "s-NL-RMM-GKS"): a block visit with fixed lambda and weights and
  a basis that reaches the image space returns the dense solution of that
  block's own problem, whatever basis and image it was started from; the
  carried compressed basis contains the image; a small streaming solve reduces
  both errors.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import nlrmm
from paper_2605_06336_gb300 import synth


def small_problem(N=16, V=12, noise=0.01, seed=0, sigma_deg=0.5):
    rng = np.random.default_rng(seed)
    g = oracle.Geometry(N, synth.n_bins(N), V)
    th_nom = np.sort(rng.uniform(0, math.pi, V))
    th_true = th_nom + rng.normal(0, math.radians(sigma_deg), V)
    u_true = synth.rasterize(N, synth.random_ellipses(N, 3, rng)).ravel()
    b_true = oracle.forward(g, th_true, u_true)
    e = rng.standard_normal(g.m)
    e *= noise * np.linalg.norm(b_true) / np.linalg.norm(e)
    return g, th_nom, th_true, u_true, b_true + e, np.linalg.norm(e)


def test_psi_is_the_kronecker_difference_operator():
    g = oracle.Geometry(7, 11, 3, views_per_frame=[1, 2])
    N = g.N
    L = sp.diags([-np.ones(N - 1), np.ones(N - 1)], [0, 1], shape=(N - 1, N))
    I = sp.identity(N)
    Psi1 = sp.vstack([sp.kron(I, L), sp.kron(L, I)])   # horizontal then vertical, row-major image
    rng = np.random.default_rng(1)
    u = rng.standard_normal(g.n)
    z = nlrmm.psi(g, u)
    U = u.reshape(g.F, N * N)
    nx = N * (N - 1)
    for f in range(g.F):
        ref = Psi1 @ U[f]
        np.testing.assert_allclose(z[f * nx:(f + 1) * nx], ref[:nx], atol=1e-14)
        np.testing.assert_allclose(z[g.F * nx + f * nx: g.F * nx + (f + 1) * nx], ref[nx:], atol=1e-14)
    y = rng.standard_normal(z.size)
    assert abs(z @ y - u @ nlrmm.psi_t(g, y)) < 1e-12 * np.linalg.norm(z) * np.linalg.norm(y)


def test_aniso_tv_is_the_space_time_kronecker_operator():
    """Psi with the temporal block equals D_1 = [I_nt (x) L_s; L_t (x) I_ns] (rows grouped
    as spatial-horizontal, spatial-vertical, temporal) and psi_t is its transpose."""
    N, F = 6, 4
    g = oracle.Geometry(N, 9, F, views_per_frame=[1] * F)
    L = lambda k: sp.diags([-np.ones(k - 1), np.ones(k - 1)], [0, 1], shape=(k - 1, k))
    I = lambda k: sp.identity(k)
    Lh = sp.kron(I(N), L(N))            # within a row-major frame: horizontal differences
    Lv = sp.kron(L(N), I(N))            # vertical differences
    D1 = sp.vstack([sp.kron(I(F), Lh), sp.kron(I(F), Lv), sp.kron(L(F), I(N * N))]).tocsr()
    rng = np.random.default_rng(2)
    u = rng.standard_normal(g.n)
    z = rng.standard_normal(D1.shape[0])
    np.testing.assert_allclose(nlrmm.psi(g, u, temporal=True), D1 @ u, atol=1e-13)
    np.testing.assert_allclose(nlrmm.psi_t(g, z, temporal=True), D1.T @ z, atol=1e-13)
    assert nlrmm.psi(g, u, temporal=True).shape[0] == 2 * F * N * (N - 1) + (F - 1) * N * N


def test_majorant_touches_and_majorizes():
    g, th, _, u_true, b, _ = small_problem(N=12, V=8)
    rng = np.random.default_rng(2)
    uk = u_true + 0.1 * rng.standard_normal(g.n)
    lam, eps = 0.7, 1e-2
    Jk = nlrmm.objective(g, th, None, uk, b, lam, eps)
    assert abs(nlrmm.majorant(g, th, None, uk, uk, b, lam, eps) - Jk) <= 1e-12 * abs(Jk)
    for _ in range(20):
        u = uk + rng.standard_normal(g.n) * rng.uniform(0.01, 2)
        assert nlrmm.majorant(g, th, None, u, uk, b, lam, eps) >= nlrmm.objective(g, th, None, u, b, lam, eps) - 1e-9


def test_reorthogonalization_survives_vectors_almost_in_the_span():
    rng = np.random.default_rng(3)
    V, _ = np.linalg.qr(rng.standard_normal((2000, 12)))
    for eps in (1e-6, 1e-9, 1e-12):
        r = V @ rng.standard_normal(12) + eps * rng.standard_normal(2000)
        q = nlrmm.cgs2(V, r)
        assert np.abs(V.T @ q).max() <= 1e-15 * np.linalg.norm(q)
        # what is removed lies in span(V): q is r minus its projection
        np.testing.assert_allclose(q, r - V @ (V.T @ r), atol=1e-13 * np.linalg.norm(r))


def test_golub_kahan_basis_spans_the_krylov_space():
    g, th, _, _, b, nn = small_problem(N=12, V=10)
    s = nlrmm.NLRMMGKS(g, b, nlrmm.Options(noise_norm=nn))
    A = oracle.dense_matrix(g, th)
    for k in (2, 3, 4, 5):
        V = s.gkb(th, k)
        K = [A.T @ b]
        for _ in range(k - 1):
            K.append(A.T @ (A @ K[-1]))
        Q, _ = np.linalg.qr(np.stack(K, 1))
        assert np.linalg.norm(V @ V.T - Q @ Q.T) <= 1e-9
        assert np.abs(V.T @ V - np.eye(k)).max() <= 1e-13
        v0 = A.T @ b
        assert abs(abs(V[:, 0] @ v0) - np.linalg.norm(v0)) <= 1e-12 * np.linalg.norm(v0)
        T = (A @ V).T @ (A @ V)
        assert np.abs(np.triu(T, 2)).max() <= 1e-12 * np.abs(T).max()


def test_full_krylov_space_gives_the_dense_solution():
    g, th, _, _, b, nn = small_problem(N=10, V=10)
    rng = np.random.default_rng(3)
    w = rng.uniform(0.5, 2.0, 2 * g.N * (g.N - 1))
    lam = 0.3
    opts = nlrmm.Options(k_min=3, k_max=3 + g.n + 5, tol1=0.0, lam_fix=lam, fixed_weights=w)
    s = nlrmm.NLRMMGKS(g, b, opts)
    V = s.gkb(th, opts.k_min)
    HV = np.stack([s.H(th, V[:, j]) for j in range(V.shape[1])], 1)
    u, *_ = s.enlarge(th, V, HV, np.zeros(g.n), opts.k_max - opts.k_min)
    A = oracle.dense_matrix(g, th)
    E = np.eye(g.n)
    PsiM = np.stack([nlrmm.psi(g, E[:, j]) for j in range(g.n)], 1)
    M = A.T @ A + lam * PsiM.T @ (w[:, None] * PsiM)
    u_ref = np.linalg.solve(M, A.T @ b)
    assert np.linalg.norm(u - u_ref) <= 1e-8 * np.linalg.norm(u_ref)


def test_fixed_lambda_enlarge_steps_decrease_the_objective():
    g, th, _, _, b, _ = small_problem(N=16, V=12, seed=4)
    lam, eps = 0.05, 1e-3
    opts = nlrmm.Options(k_min=5, k_max=25, tol1=0.0, lam_fix=lam, eps=eps)
    s = nlrmm.NLRMMGKS(g, b, opts)
    V = s.gkb(th, opts.k_min)
    HV = np.stack([s.H(th, V[:, j]) for j in range(V.shape[1])], 1)
    u = np.zeros(g.n)
    J = [nlrmm.objective(g, th, None, u, b, lam, eps)]
    for _ in range(12):
        u, _, V, HV, *_ = s.enlarge(th, V, HV, u, 1)
        J.append(nlrmm.objective(g, th, None, u, b, lam, eps))
    assert all(J[i + 1] <= J[i] * (1 + 1e-12) for i in range(len(J) - 1)), J
    assert J[-1] < 0.5 * J[0]


@pytest.mark.parametrize("k_min,k_max,iters,tol", [(3, 8, 30, 1e-10), (4, 12, 15, 1e-11)])
def test_restarted_outer_loop_converges_to_the_dense_solution(k_min, k_max, iters, tol):
    g, th, _, _, b, _ = small_problem(N=10, V=10)
    rng = np.random.default_rng(3)
    w = rng.uniform(0.5, 2.0, 2 * g.N * (g.N - 1))
    lam = 0.3
    A = oracle.dense_matrix(g, th)
    E = np.eye(g.n)
    PsiM = np.stack([nlrmm.psi(g, E[:, j]) for j in range(g.n)], 1)
    u_ref = np.linalg.solve(A.T @ A + lam * PsiM.T @ (w[:, None] * PsiM), A.T @ b)

    def J(u):
        return 0.5 * np.sum((A @ u - b) ** 2) + 0.5 * lam * np.sum(w * (PsiM @ u) ** 2)

    opts = nlrmm.Options(k_min=k_min, k_max=k_max, tol1=0.0, lam_fix=lam, fixed_weights=w,
                         update_theta=False, stop_on_convergence=False, outer_iters=iters)
    Js = []
    u, theta, _ = nlrmm.NLRMMGKS(g, b, opts).solve(th, callback=lambda it, u, *_: Js.append(J(u)))
    assert np.array_equal(theta, th)
    assert all(Js[i + 1] <= Js[i] * (1 + 1e-12) for i in range(len(Js) - 1)), Js
    assert np.linalg.norm(u - u_ref) <= tol * np.linalg.norm(u_ref)


@pytest.mark.parametrize("k_min,k_max,iters", [(3, 8, 40), (4, 12, 20)])
def test_restarted_dynamic_loop_converges_to_the_space_time_dense_solution(k_min, k_max, iters):
    rng = np.random.default_rng(5)
    N, vpf = 6, [4, 5, 3]
    g = oracle.Geometry(N, synth.n_bins(N), sum(vpf), views_per_frame=vpf)
    th = np.sort(rng.uniform(0, math.pi, g.V))
    b = oracle.forward(g, th, rng.uniform(size=g.n)) + 0.01 * rng.standard_normal(g.m)
    w = rng.uniform(0.5, 2.0, nlrmm.psi(g, np.zeros(g.n), temporal=True).size)
    lam = 0.3
    A = oracle.dense_matrix(g, th)
    E = np.eye(g.n)
    D1 = np.stack([nlrmm.psi(g, E[:, j], temporal=True) for j in range(g.n)], 1)   # pinned by the Kronecker test
    u_ref = np.linalg.solve(A.T @ A + lam * D1.T @ (w[:, None] * D1), A.T @ b)

    def J(u):
        return 0.5 * np.sum((A @ u - b) ** 2) + 0.5 * lam * np.sum(w * (D1 @ u) ** 2)

    opts = nlrmm.Options(k_min=k_min, k_max=k_max, tol1=0.0, lam_fix=lam, fixed_weights=w, update_theta=False,
                         stop_on_convergence=False, outer_iters=iters, temporal=True)
    Js = []
    u, _, _ = nlrmm.NLRMMGKS(g, b, opts).solve(th, callback=lambda it, u, *_: Js.append(J(u)))
    assert all(Js[i + 1] <= Js[i] * (1 + 1e-12) for i in range(len(Js) - 1)), Js
    assert np.linalg.norm(u - u_ref) <= 1e-10 * np.linalg.norm(u_ref)


def test_compress_keeps_u_in_the_span_and_orthonormality():
    g, th, _, _, b, nn = small_problem(N=16, V=12, seed=5)
    opts = nlrmm.Options(k_min=5, k_max=15, noise_norm=nn, tol1=0.0)
    s = nlrmm.NLRMMGKS(g, b, opts)
    V = s.gkb(th, opts.k_min)
    assert np.abs(V.T @ V - np.eye(V.shape[1])).max() < 1e-12
    HV = np.stack([s.H(th, V[:, j]) for j in range(V.shape[1])], 1)
    u, lam, Vg, _, RH, RP, used, _ = s.enlarge(th, V, HV, np.zeros(g.n), 10)
    assert np.abs(Vg.T @ Vg - np.eye(Vg.shape[1])).max() < 1e-11
    Vk = s.compress(Vg, RH, RP, used, lam, u)
    assert Vk.shape[1] == opts.k_min
    assert np.abs(Vk.T @ Vk - np.eye(Vk.shape[1])).max() < 1e-12
    assert np.linalg.norm(u - Vk @ (Vk.T @ u)) <= 1e-12 * np.linalg.norm(u)


def test_compress_keeps_the_dominant_directions():
    g, th, _, _, b, nn = small_problem(N=12, V=10, seed=5)
    rng = np.random.default_rng(9)
    w = rng.uniform(0.5, 2.0, 2 * g.N * (g.N - 1))
    lam = 0.2
    opts = nlrmm.Options(k_min=4, k_max=14, tol1=0.0, lam_fix=lam, fixed_weights=w)
    s = nlrmm.NLRMMGKS(g, b, opts)
    V = s.gkb(th, opts.k_min)
    HV = np.stack([s.H(th, V[:, j]) for j in range(V.shape[1])], 1)
    u, lam_used, Vg, _, RH, RP, used, _ = s.enlarge(th, V, HV, np.zeros(g.n), 10)
    assert lam_used == lam
    Vk = s.compress(Vg, RH, RP, used, lam, u)
    A = oracle.dense_matrix(g, th)
    E = np.eye(g.n)
    PsiM = np.stack([nlrmm.psi(g, E[:, j]) for j in range(g.n)], 1)
    Vu = Vg[:, :used]
    M = Vu.T @ (A.T @ A + lam * PsiM.T @ (w[:, None] * PsiM)) @ Vu
    ev, Q = np.linalg.eigh(M)
    keep = opts.k_min - 1
    assert ev[-keep] - ev[-keep - 1] > 1e-6 * ev[-1]          # the kept block is separated
    top = Vu @ Q[:, -keep:]
    got = Vk[:, :keep]
    assert np.linalg.norm(top @ top.T - got @ got.T) <= 1e-8


def test_discrepancy_principle_hits_the_target():
    g, th, _, _, b, nn = small_problem(N=16, V=12, seed=6, noise=0.05)
    opts = nlrmm.Options(noise_norm=nn)
    s = nlrmm.NLRMMGKS(g, b, opts)
    V = s.gkb(th, 30)
    HV = np.stack([s.H(th, V[:, j]) for j in range(V.shape[1])], 1)
    QH, RH = np.linalg.qr(HV)
    PsiV = np.stack([nlrmm.psi(g, V[:, j]) for j in range(V.shape[1])], 1)
    _, RP = np.linalg.qr(PsiV)
    QHb = QH.T @ b
    lam = s.choose_lambda(RH, RP, QHb)
    target = (opts.tau * nn) ** 2
    assert 1e-10 < lam < 1e10
    phi, y = s.projected_residual2(RH, RP, QHb, lam)
    assert abs(phi - target) <= 1e-8 * target
    # the same residual computed in the full space
    r = HV @ y - b
    assert abs(r @ r - phi) <= 1e-9 * target


def test_discrepancy_targets_out_of_reach_give_the_bracket_ends():
    """The reading for targets no lambda in [10^-10, 10^10] reaches: a target at or below
    the smallest projected residual gives 10^-10, one at or above the largest 10^10;
    phi is increasing in lambda in between."""
    g, th, _, _, b, nn = small_problem(N=16, V=12, seed=6, noise=0.05)
    s = nlrmm.NLRMMGKS(g, b, nlrmm.Options(noise_norm=nn))
    V = s.gkb(th, 8)
    HV = np.stack([s.H(th, V[:, j]) for j in range(V.shape[1])], 1)
    QH, RH = np.linalg.qr(HV)
    _, RP = np.linalg.qr(np.stack([nlrmm.psi(g, V[:, j]) for j in range(V.shape[1])], 1))
    QHb = QH.T @ b
    phis = [s.projected_residual2(RH, RP, QHb, 10.0 ** t)[0] for t in np.linspace(-10, 10, 41)]
    assert all(p1 >= p0 * (1 - 1e-12) for p0, p1 in zip(phis, phis[1:]))
    lo_phi, hi_phi = phis[0], phis[-1]
    s.o.noise_norm = 0.5 * np.sqrt(lo_phi) / s.o.tau         # target below every reachable residual
    assert s.choose_lambda(RH, RP, QHb) == 1e-10
    s.o.noise_norm = 2.0 * np.sqrt(hi_phi) / s.o.tau         # target above every reachable residual
    assert s.choose_lambda(RH, RP, QHb) == 1e10


def test_gauss_newton_reaches_the_single_view_minimizer():
    N = 24
    g = oracle.Geometry(N, synth.n_bins(N), 1)
    rng = np.random.default_rng(7)
    u = synth.rasterize(N, synth.random_ellipses(N, 4, rng)).ravel()
    th_true = np.array([0.61])
    b = oracle.forward(g, th_true, u)
    opts = nlrmm.Options(maxiter_p=1)
    s = nlrmm.NLRMMGKS(g, b, opts)
    th = th_true + math.radians(0.8)
    for _ in range(25):
        th = s.update_param(th, u)
    # brute force: golden-section search of f(theta) around the start
    f = lambda t: float(s.view_f(np.array([t]), u)[0])
    lo, hi = th_true[0] - math.radians(2), th_true[0] + math.radians(2)
    gr = (math.sqrt(5) - 1) / 2
    a, c = hi - gr * (hi - lo), lo + gr * (hi - lo)
    for _ in range(80):
        if f(a) < f(c):
            hi = c
        else:
            lo = a
        a, c = hi - gr * (hi - lo), lo + gr * (hi - lo)
    t_min = 0.5 * (lo + hi)
    assert abs(th[0] - t_min) <= 1e-6
    assert abs(th[0] - th_true[0]) <= 1e-6
    assert f(th[0]) <= f(th_true[0] + math.radians(0.8))


def test_armijo_never_increases_a_view_misfit():
    g, th_nom, th_true, u_true, b, _ = small_problem(N=20, V=15, seed=8, sigma_deg=1.0)
    s = nlrmm.NLRMMGKS(g, b, nlrmm.Options(maxiter_p=1))
    th = th_nom.copy()
    f_prev = s.view_f(th, u_true)
    for _ in range(4):
        th = s.update_param(th, u_true)
        f = s.view_f(th, u_true)
        assert np.all(f <= f_prev + 1e-12)
        f_prev = f


@pytest.mark.slow
def test_small_alternating_solve_reduces_errors():
    g, th_nom, th_true, u_true, b, nn = small_problem(N=32, V=30, seed=9, sigma_deg=0.5)
    opts = nlrmm.Options(noise_norm=nn, outer_iters=8, stop_on_convergence=False)
    s = nlrmm.NLRMMGKS(g, b, opts)
    u, th, hist = s.solve(th_nom, u_true=u_true, theta_true=th_true)
    e0 = np.linalg.norm(th_nom - th_true)
    assert np.linalg.norm(th - th_true) < 0.5 * e0
    assert hist.rre[-1] < hist.rre[0]
    assert hist.rre[-1] < 0.5


def test_varpro_reduced_gradient_matches_central_differences():
    # smooth image and a basis of smooth vectors: few interpolation kinks change slope
    g, th_nom, th_true, u_true, b, nn = small_problem(N=20, V=14, seed=11)
    s = nlrmm.NLRMMGKS(g, b, nlrmm.Options(noise_norm=nn))
    V = s.gkb(th_nom, 6)
    rng = np.random.default_rng(12)
    w = rng.uniform(0.5, 2.0, 2 * g.N * (g.N - 1))
    lam = 0.2
    grad, f0, _ = nlrmm.varpro_gradient(g, b, th_nom, V, lam, w)
    errs = {}
    for h in (1e-4, 1e-5, 1e-6):
        err = ref = 0.0
        for _ in range(8):
            d = rng.standard_normal(g.V)
            fp = nlrmm.varpro_objective(g, b, th_nom + h * d, V, lam, w)[0]
            fm = nlrmm.varpro_objective(g, b, th_nom - h * d, V, lam, w)[0]
            err += abs((fp - fm) / (2 * h) - grad @ d)
            ref += abs(grad @ d)
        errs[h] = err / ref
    assert errs[1e-4] < 5e-2, errs
    assert errs[1e-6] < max(errs[1e-4] / 20, 1e-7), errs


def _varpro_case(N=20, V=14, k=6, seed=11):
    g, th_nom, th_true, u_true, b, nn = small_problem(N=N, V=V, seed=seed)
    s = nlrmm.NLRMMGKS(g, b, nlrmm.Options(noise_norm=nn))
    Vb = s.gkb(th_nom, k)
    rng = np.random.default_rng(seed + 1)
    w = rng.uniform(0.5, 2.0, 2 * g.N * (g.N - 1))
    return g, th_nom, th_true, b, Vb, w, rng


def _reduced_residuals(g, b, theta, Vb, lam, w):
    _, _, u = nlrmm.varpro_objective(g, b, theta, Vb, lam, w)
    return oracle.forward(g, theta, u) - b, np.sqrt(w) * nlrmm.psi(g, u)


def test_varpro_sensitivity_jacobians_match_central_differences():
    g, th, _, b, Vb, w, rng = _varpro_case()
    lam = 0.2
    Jr, Js, r, s, f, u = nlrmm.varpro_jacobians(g, b, th, Vb, lam, w)
    r0, s0 = _reduced_residuals(g, b, th, Vb, lam, w)
    assert np.allclose(r, r0, rtol=0, atol=1e-12 * np.linalg.norm(r0))
    assert np.allclose(s, s0, rtol=0, atol=1e-12 * np.linalg.norm(s0))
    errs = {}
    for h in (1e-4, 1e-5, 1e-6):
        er = es = nr = ns = 0.0
        for _ in range(6):
            d = rng.standard_normal(g.V)
            rp, sp_ = _reduced_residuals(g, b, th + h * d, Vb, lam, w)
            rm, sm = _reduced_residuals(g, b, th - h * d, Vb, lam, w)
            er += np.linalg.norm((rp - rm) / (2 * h) - Jr @ d)
            es += np.linalg.norm((sp_ - sm) / (2 * h) - Js @ d)
            nr += np.linalg.norm(Jr @ d)
            ns += np.linalg.norm(Js @ d)
        errs[h] = (er / nr, es / ns)
    # interpolation kinks make the quotients inexact by an error that shrinks with h
    assert max(errs[1e-4]) < 5e-2, errs
    assert errs[1e-6][0] < max(errs[1e-4][0] / 20, 1e-7), errs
    assert errs[1e-6][1] < max(errs[1e-4][1] / 20, 1e-7), errs


def test_varpro_jacobians_with_temporal_differences_match_central_differences():
    """The same pin with ANISO-TV (frame-to-frame differences in Psi) on 3 frames."""
    rng = np.random.default_rng(13)
    N, vpf = 14, [5, 4, 5]
    g = oracle.Geometry(N, synth.n_bins(N), sum(vpf), vpf)
    th = np.sort(synth.random_angles(g.V, rng))
    u = np.stack([synth.rasterize(N, synth.random_ellipses(N, 2, rng)) for _ in vpf]).ravel()
    b = oracle.forward(g, th, u) + 0.01 * rng.standard_normal(g.m)
    Vb, _ = np.linalg.qr(rng.standard_normal((g.n, 5)))
    ne = nlrmm.psi(g, u, True).size
    w = rng.uniform(0.5, 2.0, ne)
    lam = 0.3
    Jr, Js, r, s_, f, uu = nlrmm.varpro_jacobians(g, b, th, Vb, lam, w, None, True)
    errs = {}
    for h in (1e-4, 1e-6):
        er = nr = 0.0
        for _ in range(4):
            d = rng.standard_normal(g.V)
            up = nlrmm.varpro_objective(g, b, th + h * d, Vb, lam, w, None, True)[2]
            um = nlrmm.varpro_objective(g, b, th - h * d, Vb, lam, w, None, True)[2]
            sp_, sm = np.sqrt(w) * nlrmm.psi(g, up, True), np.sqrt(w) * nlrmm.psi(g, um, True)
            er += np.linalg.norm((sp_ - sm) / (2 * h) - Js @ d)
            nr += np.linalg.norm(Js @ d)
        errs[h] = er / nr
    assert errs[1e-6] < max(errs[1e-4] / 20, 1e-7), errs


def test_varpro_gauss_newton_gradient_is_the_envelope_gradient():
    g, th, _, b, Vb, w, _ = _varpro_case(N=16, V=10, k=5, seed=21)
    lam = 0.5
    Jr, Js, r, s, f, u = nlrmm.varpro_jacobians(g, b, th, Vb, lam, w)
    ge, fe, _ = nlrmm.varpro_gradient(g, b, th, Vb, lam, w)
    gj = Jr.T @ r + lam * (Js.T @ s)
    assert abs(f - fe) <= 1e-14 * fe
    assert np.linalg.norm(gj - ge) <= 1e-9 * np.linalg.norm(ge)


def test_varpro_gauss_newton_converges_quadratically_to_the_true_angles():
    """Noise-free data, the true image in span(V), lambda ~ 0: the reduced
    residual vanishes at the true angles, where Gauss-Newton converges
    quadratically (a diagonal or otherwise wrong Gauss-Newton matrix converges
    linearly: its error after 3 steps is ~1e-5 rad here)."""
    N, Vn, k = 16, 8, 6
    rng = np.random.default_rng(5)
    g = oracle.Geometry(N, synth.n_bins(N), Vn)
    th_true = np.sort(rng.uniform(0, math.pi, Vn))
    u_true = synth.rasterize(N, synth.random_ellipses(N, 3, rng)).ravel()
    b = oracle.forward(g, th_true, u_true)
    Vb, _ = np.linalg.qr(np.column_stack([u_true, rng.standard_normal((g.n, k - 1))]))
    lam, w = 1e-10, np.ones(2 * N * (N - 1))
    th = th_true + rng.normal(0, math.radians(0.5), Vn)
    s = nlrmm.NLRMMGKS(g, b, nlrmm.Options(maxiter_p=1))
    f_prev = nlrmm.varpro_objective(g, b, th, Vb, lam, w)[0]
    errs = []
    for _ in range(4):
        th = s.update_param_varpro(th, Vb, lam, w)
        f = nlrmm.varpro_objective(g, b, th, Vb, lam, w)[0]
        assert f <= f_prev + 1e-15
        f_prev = f
        errs.append(float(np.max(np.abs(th - th_true))))
    assert errs[2] <= 1e-9, errs
    assert errs[1] <= 10 * errs[0] ** 2 / math.radians(0.5) + 1e-10, errs


def test_small_varpro_solve_reduces_errors():
    g, th_nom, th_true, u_true, b, nn = small_problem(N=24, V=20, seed=9, sigma_deg=0.5)
    opts = nlrmm.Options(noise_norm=nn, outer_iters=5, stop_on_convergence=False, varpro=True)
    u, th, hist = nlrmm.NLRMMGKS(g, b, opts).solve(th_nom, u_true=u_true, theta_true=th_true)
    assert np.linalg.norm(th - th_true) < 0.5 * np.linalg.norm(th_nom - th_true)
    assert hist.rre[-1] < hist.rre[0]


def _blocks(g, th, b, nblocks, opts_for):
    """Split the views of (g, th, b) into nblocks consecutive blocks."""
    idx = np.array_split(np.arange(g.V), nblocks)
    bv = b.reshape(g.V, g.B)
    out = []
    for j, ix in enumerate(idx):
        gj = oracle.Geometry(g.N, g.B, len(ix))
        out.append((nlrmm.NLRMMGKS(gj, bv[ix].ravel(), opts_for(j, ix)), th[ix]))
    return out


def test_stream_visit_solves_its_own_block_problem():
    g, th, _, _, b, _ = small_problem(N=10, V=10, seed=21)
    rng = np.random.default_rng(22)
    w = rng.uniform(0.5, 2.0, 2 * g.N * (g.N - 1))
    lam = 0.3
    opts = lambda j, ix: nlrmm.Options(k_min=3, k_max=3 + g.n + 5, tol1=0.0, lam_fix=lam, fixed_weights=w,
                                       update_theta=False, stop_on_convergence=False)
    blocks = _blocks(g, th, b, 2, opts)
    E = np.eye(g.n)
    PsiM = np.stack([nlrmm.psi(g, E[:, j]) for j in range(g.n)], 1)
    seen = []

    def cb(p, j, u, V, thetas):
        blk, thj = blocks[j]
        A = oracle.dense_matrix(blk.g, thj)
        M = A.T @ A + lam * PsiM.T @ (w[:, None] * PsiM)
        u_ref = np.linalg.solve(M, A.T @ blk.b)
        seen.append(np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref))

    nlrmm.stream_solve([s for s, _ in blocks], [t for _, t in blocks], passes=2, callback=cb)
    assert len(seen) == 4 and max(seen) <= 1e-8, seen


def test_stream_carries_the_image_in_the_basis():
    g, th, _, _, b, nn = small_problem(N=16, V=12, seed=23)
    opts = lambda j, ix: nlrmm.Options(k_min=5, k_max=15, noise_norm=nn / math.sqrt(3), stop_on_convergence=False)
    blocks = _blocks(g, th, b, 3, opts)
    checks = []

    def cb(p, j, u, V, thetas):
        checks.append((np.linalg.norm(u - V @ (V.T @ u)) / np.linalg.norm(u), np.abs(V.T @ V - np.eye(V.shape[1])).max(),
                       V.shape[1]))

    nlrmm.stream_solve([s for s, _ in blocks], [t for _, t in blocks], passes=2, callback=cb)
    assert len(checks) == 6
    for resid, orth, k in checks:
        assert resid <= 1e-12 and orth <= 1e-12 and k == 5


@pytest.mark.slow
def test_small_streaming_solve_reduces_errors():
    rng = np.random.default_rng(24)
    N, V, nb = 32, 30, 3
    g = oracle.Geometry(N, synth.n_bins(N), V)
    th_nom = np.sort(rng.uniform(0, math.pi, V))
    th_true = th_nom + rng.normal(0, math.radians(0.5), V)
    perm = rng.permutation(V)  # views drawn into blocks without replacement
    u_true = synth.rasterize(N, synth.random_ellipses(N, 3, rng)).ravel()
    b_true = oracle.forward(g, th_true, u_true).reshape(V, -1)
    e = rng.standard_normal(b_true.shape)
    e *= 0.01 * np.linalg.norm(b_true) / np.linalg.norm(e)
    blocks, th0, tht = [], [], []
    for ix in np.array_split(perm, nb):
        ix = np.sort(ix)
        gj = oracle.Geometry(N, g.B, len(ix))
        o = nlrmm.Options(noise_norm=float(np.linalg.norm(e[ix])), stop_on_convergence=False)
        blocks.append(nlrmm.NLRMMGKS(gj, (b_true[ix] + e[ix]).ravel(), o))
        th0.append(th_nom[ix])
        tht.append(th_true[ix])
    u, th, hist = nlrmm.stream_solve(blocks, th0, passes=6, u_true=u_true, theta_true=tht)
    err0 = np.linalg.norm(np.concatenate(th0) - np.concatenate(tht))
    assert np.linalg.norm(np.concatenate(th) - np.concatenate(tht)) < 0.6 * err0
    assert all(hist.rre[i + 1] <= hist.rre[i] for i in range(len(hist.rre) - 1)), hist.rre
    assert hist.rre[-1] < 0.5 * hist.rre[0]


@pytest.mark.slow
def test_aniso_tv_helps_a_slowly_moving_sequence():
    """Few views per frame of a slowly translating phantom: coupling the frames
    through D_1 (ANISO-TV) gives a lower reconstruction error than spatial
    differences alone (the motivation of the dynamic extension)."""
    rng = np.random.default_rng(41)
    N, F, vpf = 24, 4, [6, 7, 6, 7]
    ells = synth.random_ellipses(N, 3, rng)
    frames = [synth.rasterize(N, ells, shift=(0.5 * f, 0.0)) for f in range(F)]
    u_true = np.stack(frames).ravel()
    V = sum(vpf)
    g = oracle.Geometry(N, synth.n_bins(N), V, views_per_frame=vpf)
    th = np.sort(rng.uniform(0, math.pi, V))
    b_true = oracle.forward(g, th, u_true)
    e = rng.standard_normal(g.m)
    e *= 0.01 * np.linalg.norm(b_true) / np.linalg.norm(e)
    rre = {}
    for tm in (False, True):
        o = nlrmm.Options(noise_norm=float(np.linalg.norm(e)), outer_iters=6, stop_on_convergence=False,
                          update_theta=False, temporal=tm)
        u, _, hist = nlrmm.NLRMMGKS(g, b_true + e, o).solve(th, u_true=u_true)
        rre[tm] = hist.rre[-1]
    assert rre[True] < rre[False], rre


def _view_minimizers(s, th0, u, halfwidth):
    """Per-view golden-section minimizers of the separable view misfits f_v(theta_v)."""
    V = th0.size
    lo, hi = th0 - halfwidth, th0 + halfwidth
    gr = (math.sqrt(5) - 1) / 2
    for _ in range(70):
        a, c = hi - gr * (hi - lo), lo + gr * (hi - lo)
        fa, fc = s.view_f(a, u), s.view_f(c, u)
        left = fa < fc
        hi = np.where(left, c, hi)
        lo = np.where(left, lo, a)
    return 0.5 * (lo + hi)


def test_armijo_noise_floor_ends_rounding_decided_searches():
    # noisy data: at a view's own minimizer its predicted decrease c1 |g d| is far
    # below the rounding of f_v, so any Armijo decision there is rounding noise
    g, th_nom, th_true, u_true, b, _ = small_problem(N=20, V=16, seed=21, sigma_deg=1.0)
    s = nlrmm.NLRMMGKS(g, b, nlrmm.Options(maxiter_p=1))
    th_star = _view_minimizers(s, th_true, u_true, math.radians(3.0))
    near = np.arange(16) < 8                  # views 0..7 at their minimizer, 8..15 half a degree off
    th0 = np.where(near, th_star, th_star + math.radians(0.5))
    grad, jn2, f0, rho = s.view_terms(th0, u_true)
    d = -grad / (jn2 + 1e-8 * jn2.max())
    u32 = 2.0 ** -24
    pred = np.abs(grad * d) / rho
    assert np.all(pred[near] < u32) and np.all(pred[~near] > 1e3 * u32)
    assert np.all(rho >= 2 * f0)   # |H u| + |b| >= |r| term by term

    s_off = nlrmm.NLRMMGKS(g, b, nlrmm.Options(maxiter_p=1, armijo_eps=0.0))
    th_off = s_off.update_param(th0, u_true)
    trials_off = s_off.last_trials
    s_on = nlrmm.NLRMMGKS(g, b, nlrmm.Options(maxiter_p=1, armijo_eps=u32))
    th_on = s_on.update_param(th0, u_true)
    trials_on = s_on.last_trials
    # without the floor the searches at the minimizers run (rounding decides them);
    # with it they end before the first trial and the angles stay
    assert trials_off[near].sum() > 8
    assert np.all(trials_on[near] == 0)
    assert np.array_equal(th_on[near], th0[near])
    # views with a real decrease take exactly the steps they take without the floor
    assert np.array_equal(th_on[~near], th_off[~near])
    assert np.array_equal(trials_on[~near], trials_off[~near])
    f_on = s.view_f(th_on, u_true)
    assert np.all(f_on[~near] < f0[~near])
    # the floor at FP64 rounding still ends the searches at the minimizers
    s64 = nlrmm.NLRMMGKS(g, b, nlrmm.Options(maxiter_p=1))
    s64.update_param(th0, u_true)
    assert np.all(s64.last_trials[near] <= trials_off[near])


def test_armijo_noise_floor_stops_after_the_halving_that_crosses_it():
    # one view, a search that fails at alpha0 = 64 (a step far too long): the
    # floor at armijo_eps = alpha0 |g d| / (rho * 2^(k + 1/2)) permits trials at
    # alpha = alpha0, alpha0 / 2, ..., alpha0 2^-k and none after
    g, th_nom, th_true, u_true, b, _ = small_problem(N=20, V=1, seed=22, sigma_deg=1.0)
    opts = nlrmm.Options(maxiter_p=1, alpha0=64.0, armijo_eps=0.0)
    s = nlrmm.NLRMMGKS(g, b, opts)
    th0 = th_true + math.radians(0.4)
    s.update_param(th0, u_true)
    t_free = int(s.last_trials[0])
    assert t_free >= 5                           # alpha0 = 64 overshoots: several halvings needed
    grad, jn2, f0, rho = s.view_terms(th0, u_true)
    d = -grad / (jn2 + 1e-8 * jn2.max())
    for k in range(t_free - 1):
        opts_k = nlrmm.Options(maxiter_p=1, alpha0=64.0,
                               armijo_eps=64.0 * abs(grad[0] * d[0]) / (rho[0] * 2.0 ** (k + 0.5)))
        s_k = nlrmm.NLRMMGKS(g, b, opts_k)
        th_k = s_k.update_param(th0, u_true)
        assert int(s_k.last_trials[0]) == k + 1
        assert th_k[0] == th0[0]                 # no trial accepted before the floor: no step


def test_rounding_scale_bounds_the_float32_misfit_error():
    # rho_v = sum_b |r_b| (|(Hu)_b| + |b_b|) bounds, to first order, the error of
    # evaluating f_v = 1/2 |r_v|^2 from float32 residuals: each r_b = fl(fl(Hu) - fl(b))
    # is off by at most u (|Hu| + |b| + |r|) <= 2u (|Hu| + |b|), so |f32 - f| <= 2 u rho
    g, th_nom, th_true, u_true, b, _ = small_problem(N=24, V=20, seed=23, sigma_deg=1.0)
    s = nlrmm.NLRMMGKS(g, b, nlrmm.Options())
    _, _, f, rho = s.view_terms(th_nom, u_true)
    Hu = oracle.forward(g, th_nom, u_true).reshape(g.V, g.B)
    r32 = (Hu.astype(np.float32) - b.reshape(g.V, g.B).astype(np.float32)).astype(np.float64)
    f32 = 0.5 * (r32 * r32).sum(1)
    u32 = 2.0 ** -24
    ratio = np.abs(f32 - f) / (u32 * rho)
    assert np.all(ratio <= 2.0 + 1e-6), ratio.max()
    assert ratio.max() > 1e-3          # and rho is not a vacuous bound
    assert np.all(rho >= 2 * f)


def test_shared_offset_update_reaches_the_minimizer_over_the_offset():
    # every view shifted by one offset p_true (the scalar parameter of the paper's
    # CT experiments); noise-free data and the true image: the Gauss-Newton
    # update on p (gradient sum_v g_v, matrix sum_v |J_v|^2) reaches the
    # brute-force minimizer of F(p) = sum_v f_v(theta_nom + p), which is p_true
    N, V = 24, 14
    g = oracle.Geometry(N, synth.n_bins(N), V)
    rng = np.random.default_rng(31)
    u = synth.rasterize(N, synth.random_ellipses(N, 4, rng)).ravel()
    th_nom = np.sort(rng.uniform(0, math.pi, V))
    p_true = math.radians(0.7)
    b = oracle.forward(g, th_nom + p_true, u)
    s = nlrmm.NLRMMGKS(g, b, nlrmm.Options(maxiter_p=1, shared_offset=True))
    th = th_nom.copy()
    for _ in range(30):
        th = s.update_param_shared(th, u)
    shift = th - th_nom
    assert np.ptp(shift) <= 1e-15                         # one offset for every view
    F = lambda p: float(s.view_f(th_nom + p, u).sum())
    lo, hi = p_true - math.radians(2), p_true + math.radians(2)
    gr = (math.sqrt(5) - 1) / 2
    a, c = hi - gr * (hi - lo), lo + gr * (hi - lo)
    for _ in range(80):
        if F(a) < F(c):
            hi = c
        else:
            lo = a
        a, c = hi - gr * (hi - lo), lo + gr * (hi - lo)
    assert abs(shift[0] - 0.5 * (lo + hi)) <= 1e-7
    assert abs(shift[0] - p_true) <= 1e-7
    # the gradient it steps on is that of F: J 1 summed over the views
    grad, _, _, _ = s.view_terms(th_nom, u)
    h = 1e-6
    assert abs(grad.sum() - (F(h) - F(-h)) / (2 * h)) <= 2e-3 * abs(grad.sum())


@pytest.mark.slow
def test_small_solve_with_a_shared_offset_keeps_one_offset():
    # a common shift of every angle is equivalent to rotating the image, so the
    # reconstruction absorbs most of it and the alternating solve recovers it
    # slowly (with the true image one update recovers it, see above); what the
    # solve must do: keep one offset for all views, move it towards p_true, and
    # lower the image error
    N, V = 32, 30
    rng = np.random.default_rng(32)
    g = oracle.Geometry(N, synth.n_bins(N), V)
    th_nom = np.sort(rng.uniform(0, math.pi, V))
    p_true = math.radians(0.8)
    u_true = synth.rasterize(N, synth.random_ellipses(N, 3, rng)).ravel()
    b_true = oracle.forward(g, th_nom + p_true, u_true)
    e = rng.standard_normal(g.m)
    e *= 0.01 * np.linalg.norm(b_true) / np.linalg.norm(e)
    opts = nlrmm.Options(noise_norm=float(np.linalg.norm(e)), outer_iters=8, stop_on_convergence=False,
                         shared_offset=True)
    u, th, hist = nlrmm.NLRMMGKS(g, b_true + e, opts).solve(th_nom, u_true=u_true)
    shift = th - th_nom
    assert np.ptp(shift) <= 1e-14
    assert 0.05 * p_true < shift[0] < p_true
    assert hist.rre[-1] < hist.rre[0]
    with pytest.raises(ValueError):
        nlrmm.NLRMMGKS(g, b_true + e, nlrmm.Options(noise_norm=1.0, shared_offset=True, varpro=True)).param_update(
            th_nom, u_true, None, 1.0)
