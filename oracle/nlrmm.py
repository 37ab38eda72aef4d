"""FP64 reference of the NL-RMM-GKS solver (AltMin form), written step by step.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Uses the oracle
operators of this package and numpy's QR / SVD / solve as library steps.

Passages followed:
  * MM weights P = diag((z^2 + eps^2)^(-1/4)), z = Psi u, and the quadratic
    majorant (Eq. (3.1)-(3.2), Sec. 3.1);
  * generalized Krylov projection: QR of H V and P Psi V, the reduced
    problem (Eq. (3.4)-(3.5)), the normal-equation residual appended to V
    (Eq. (3.6)-(3.7));
  * Alg. "Enlarge" and Alg. "Compress" (supplementary Sec. S1.2) and
    Alg. "RMM-GKS" (Sec. 3.3);
  * Alg. "UPDATE-PARAM" (damped Gauss-Newton + Armijo backtracking, Sec. 4.1.2);
  * Alg. "UPDATE-PARAM-VarPro" (Sec. 4.2): the reduced objective on the
    compressed basis, its Gauss-Newton system (J_r^T J_r + lambda J_s^T J_s)
    with Jacobian columns from the sensitivity equation, Armijo on the reduced
    objective (``varpro_jacobians``, ``NLRMMGKS.update_param_varpro``);
  * Alg. "NL-RMM-GKS" (Sec. 4.3) without the optional high-lambda solve;
  * Alg. "s-NL-RMM-GKS" (Sec. 5) over blocks of views (``stream_solve``);
  * the dynamic form with ANISO-TV (operator D_1, Alg. "Dynamic NL-RMM-GKS"): Psi gains the
    differences of consecutive frames (``Options.temporal``).

Readings where the paper is silent (also listed in the design notes):
  * Psi = forward differences without wrap, horizontal then vertical, per frame;
  * eps = 1e-3; tol_1 = 1e-3;
  * lambda by the discrepancy principle on the projected problem:
    ||H V y(lambda) - b||^2 = (tau * noise_norm)^2, tau = 1.01, bisection in
    log10(lambda) over [-10, 10] with 60 halvings; if the target is below the
    smallest reachable residual lambda = 1e-10, if above the largest 1e10;
  * GKB start vector b, k_min steps, each new right vector reorthogonalized
    twice against the previous ones;
  * one Enlarge + Compress per outer iteration; Enlarge starts from the basis
    carried over (k_min + 1 columns after the residual append) and stops after
    s = k_max - k_min steps or when ||u_new - u_old|| <= tol_1 ||u_old||;
  * Compress uses the columns of V that R_H, R_Psi were formed from (the last
    appended residual has no R entry yet): top k_min - 1 right singular
    vectors of [R_H; sqrt(lambda) R_Psi], then the normalized part of u
    orthogonal to them (skipped if it vanishes);
  * per-view angles make J^T J diagonal: the Gauss-Newton step is per view,
    d_v = -g_v / (|J_v|^2 + mu) with mu = 1e-8 max_v |J_v|^2, and the Armijo
    backtracking (c1 = 1e-4, beta = 1/2, alpha_bar = 1, at most 20 halvings,
    no step if none is accepted) is applied to each view's own data term;
    3 Gauss-Newton iterations per outer iteration;
  * Armijo in finite precision (the paper's descent lemmas assume exact
    arithmetic): before each trial, a search whose first-order change of the
    misfit, alpha * |g^T d|, is below armijo_eps * rho ends with no acceptable
    step.  rho = sum_b |r_b| (|(H u)_b| + |b_b|) over the residuals r = H u - b
    the misfit f = 1/2 |r|^2 is formed from bounds the rounding error of
    evaluating f (each r_b is off by at most a unit roundoff of |H u| + |b|),
    and armijo_eps is the unit roundoff of the precision f is computed in:
    2^-53 for FP64, 2^-24 to follow FP32 residuals.  Per view in UPDATE-PARAM
    (r of that view), on the data residual of the reduced objective in the
    VarPro update.  Such a test compares two misfits that differ by less than
    their own rounding, so its outcome carries no information;
  * shared angle offset (Options.shared_offset, the scalar parameter of the
    paper's CT experiments, Sec. 6.2, and of its dynamic CT, where one offset
    serves every frame): theta_v = theta_v^0 + p for all views; the
    Gauss-Newton step on p uses g = sum_v g_v (the gradient along the
    direction 1) and J^T J = sum_v |J_v|^2, damped by mu = mu_rel J^T J,
    with the Armijo test and its noise floor on the total misfit (rho summed
    over the views); no accepted step ends the update with the offset kept;
    not combined with the VarPro update;
  * VarPro (Options.varpro): the basis is the compressed V^(k+1)_kmin of the
    primary solve, lambda_hat = lambda^(k), B_hat = P Psi V with P^2 the MM
    weights of u^(k+1); the Gauss-Newton matrix is damped by mu = 1e-8 times
    its largest diagonal entry; the Armijo test is on the whole reduced
    objective (the views are coupled through y); when no step is accepted
    the angles stay and the remaining Gauss-Newton iterations are skipped;
    u^(k+1) stays the image of the outer iteration;
  * the residual appended at the end of an outer iteration uses the operator
    of that iteration's angles (H_k of Alg. "NL-RMM-GKS");
  * u^(0) = 0; the relative-change tests are skipped while ||u_old|| = 0;
  * outer stop: ||du|| / ||u|| < tol_u and ||dtheta|| < tol_p, or the
    iteration limit.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import Geometry, adjoint, dsample, forward, jac, jacT


# ---------------------------------------------------------------------------
# regularization operator Psi (finite differences, Sec. 2.2)
# ---------------------------------------------------------------------------
def psi(g: Geometry, u: np.ndarray, temporal: bool = False) -> np.ndarray:
    """Psi u: forward differences within each frame (horizontal block, then
    vertical); with ``temporal`` also the difference of consecutive frames
    (ANISO-TV: the operator D_1 = [I_nt (x) L_s; L_t (x) I_ns] of the dynamic
    extension, Alg. "Dynamic NL-RMM-GKS")."""
    U = u.reshape(g.F, g.N, g.N)
    dx = U[:, :, 1:] - U[:, :, :-1]
    dy = U[:, 1:, :] - U[:, :-1, :]
    parts = [dx.ravel(), dy.ravel()]
    if temporal and g.F > 1:
        parts.append((U[1:] - U[:-1]).ravel())
    return np.concatenate(parts)


def psi_t(g: Geometry, z: np.ndarray, temporal: bool = False) -> np.ndarray:
    F, N = g.F, g.N
    nx = F * N * (N - 1)
    dx = z[:nx].reshape(F, N, N - 1)
    dy = z[nx:2 * nx].reshape(F, N - 1, N)
    U = np.zeros((F, N, N))
    U[:, :, 1:] += dx
    U[:, :, :-1] -= dx
    U[:, 1:, :] += dy
    U[:, :-1, :] -= dy
    if temporal and F > 1:
        dt = z[2 * nx:].reshape(F - 1, N, N)
        U[1:] += dt
        U[:-1] -= dt
    return U.ravel()


def mm_weights(z: np.ndarray, eps: float) -> np.ndarray:
    """Diagonal of P^2 = (z^2 + eps^2)^(-1/2) (P itself has exponent -1/4)."""
    return 1.0 / np.sqrt(z * z + eps * eps)


def objective(g, theta, delta, u, b, lam, eps, temporal=False):
    """J_{eps,lambda}(u, theta) = 1/2 ||H u - b||^2 + lambda sum sqrt((Psi u)^2 + eps^2)."""
    r = forward(g, theta, u, delta) - b
    z = psi(g, u, temporal)
    return 0.5 * r @ r + lam * np.sum(np.sqrt(z * z + eps * eps))


def majorant(g, theta, delta, u, uk, b, lam, eps, temporal=False):
    """Q(u | u_k): the quadratic majorant of J_{eps,lambda} at u_k (Eq. (3.2)), constant included."""
    r = forward(g, theta, u, delta) - b
    zk = psi(g, uk, temporal)
    sk = np.sqrt(zk * zk + eps * eps)
    z = psi(g, u, temporal)
    # sqrt(t^2 + eps^2) <= sk + (t^2 - zk^2) / (2 sk) by concavity of sqrt
    return 0.5 * r @ r + lam * np.sum(sk + (z * z - zk * zk) / (2 * sk))


def cgs2(V: np.ndarray, r: np.ndarray) -> np.ndarray:
    """r - V V^T r, applied twice (classical Gram-Schmidt with reorthogonalization)."""
    if V.shape[1] == 0:
        return r
    r = r - V @ (V.T @ r)
    return r - V @ (V.T @ r)


@dataclass
class Options:
    k_min: int = 5
    k_max: int = 25
    eps: float = 1e-3
    tol1: float = 1e-3
    tau: float = 1.01
    noise_norm: float | None = None
    lam_fix: float | None = None
    lam_lo: float = -10.0
    lam_hi: float = 10.0
    lam_iters: int = 60
    maxiter_p: int = 3
    c1: float = 1e-4
    beta: float = 0.5
    alpha0: float = 1.0
    max_halvings: int = 20
    armijo_eps: float = 2.0 ** -53            # unit roundoff of the misfit's precision (Armijo noise floor)
    mu_rel: float = 1e-8
    outer_iters: int = 20
    tol_u: float = 1e-3
    tol_p: float = 1e-4
    update_theta: bool = True
    stop_on_convergence: bool = True
    fixed_weights: np.ndarray | None = None   # freeze P^2 (pins only)
    temporal: bool = False                    # ANISO-TV: add frame-to-frame differences to Psi
    varpro: bool = False                      # parameter update by Alg. "UPDATE-PARAM-VarPro"
    shared_offset: bool = False               # one angle offset shared by every view (theta^0 + p)


@dataclass
class History:
    lam: list = field(default_factory=list)
    rre: list = field(default_factory=list)
    angle_err: list = field(default_factory=list)
    du: list = field(default_factory=list)
    dtheta: list = field(default_factory=list)
    enlarge_steps: list = field(default_factory=list)
    objective: list = field(default_factory=list)


class NLRMMGKS:
    """Alternating NL-RMM-GKS on the oracle operator."""

    def __init__(self, g: Geometry, b: np.ndarray, opts: Options, delta=None):
        self.g, self.b, self.o, self.delta = g, np.asarray(b, float), opts, delta
        self.bnorm2 = float(self.b @ self.b)

    # -- operator wrappers ------------------------------------------------
    def H(self, theta, x):
        return forward(self.g, theta, x, self.delta)

    def HT(self, theta, y):
        return adjoint(self.g, theta, y, self.delta)

    # -- lambda by the discrepancy principle on the projected problem -------
    def projected_residual2(self, RH, RP, QHb, lam):
        M = RH.T @ RH + lam * (RP.T @ RP)
        y = np.linalg.solve(M, RH.T @ QHb)
        out = RH @ y - QHb
        return out @ out + (self.bnorm2 - QHb @ QHb), y

    def choose_lambda(self, RH, RP, QHb):
        o = self.o
        if o.lam_fix is not None:
            return o.lam_fix
        target = (o.tau * o.noise_norm) ** 2
        lo, hi = o.lam_lo, o.lam_hi
        if self.projected_residual2(RH, RP, QHb, 10.0 ** lo)[0] >= target:
            return 10.0 ** lo
        if self.projected_residual2(RH, RP, QHb, 10.0 ** hi)[0] <= target:
            return 10.0 ** hi
        for _ in range(o.lam_iters):
            mid = 0.5 * (lo + hi)
            if self.projected_residual2(RH, RP, QHb, 10.0 ** mid)[0] < target:
                lo = mid
            else:
                hi = mid
        return 10.0 ** (0.5 * (lo + hi))

    # -- initial basis: Golub-Kahan bidiagonalization ----------------------
    def gkb(self, theta, k):
        b = self.b
        u = b / np.linalg.norm(b)
        v = self.HT(theta, u)
        alpha = np.linalg.norm(v)
        v = v / alpha
        V = [v]
        for _ in range(1, k):
            p = self.H(theta, v) - alpha * u
            beta = np.linalg.norm(p)
            u = p / beta
            q = self.HT(theta, u) - beta * v
            q = cgs2(np.stack(V, 1), q)
            alpha = np.linalg.norm(q)
            v = q / alpha
            V.append(v)
        return np.stack(V, 1)

    # -- Alg. "Enlarge" -----------------------------------------------------
    def enlarge(self, theta, V, HV, u0, s):
        o, g, b = self.o, self.g, self.b
        u_old = u0
        lam = None
        RH = RP = None
        steps = 0
        for _ in range(s):
            w = o.fixed_weights if o.fixed_weights is not None else mm_weights(psi(g, u_old, o.temporal), o.eps)
            p = np.sqrt(w)
            QH, RH = np.linalg.qr(HV)
            PsiV = np.stack([psi(g, V[:, j], o.temporal) for j in range(V.shape[1])], 1)
            _, RP = np.linalg.qr(p[:, None] * PsiV)
            QHb = QH.T @ b
            lam = self.choose_lambda(RH, RP, QHb)
            y = np.linalg.solve(RH.T @ RH + lam * (RP.T @ RP), RH.T @ QHb)
            u = V @ y
            r = self.HT(theta, self.H(theta, u) - b) + lam * psi_t(g, w * psi(g, u, o.temporal), o.temporal)
            r = cgs2(V, r)
            nr = np.linalg.norm(r)
            steps += 1
            used = V.shape[1]
            if nr > 0:
                vn = r / nr
                V = np.concatenate([V, vn[:, None]], 1)
                HV = np.concatenate([HV, self.H(theta, vn)[:, None]], 1)
            nu = np.linalg.norm(u_old)
            stop = nr == 0 or (nu > 0 and np.linalg.norm(u - u_old) <= o.tol1 * nu)
            u_old = u
            if stop:
                break
        return u_old, lam, V, HV, RH, RP, used, steps

    # -- Alg. "Compress" ------------------------------------------------------
    def compress(self, V, RH, RP, used, lam, u):
        k_min = self.o.k_min
        M = np.vstack([RH, np.sqrt(lam) * RP])
        _, _, Wt = np.linalg.svd(M, full_matrices=False)
        W = Wt[: k_min - 1].T
        Vt = V[:, :used] @ W
        un = u - Vt @ (Vt.T @ u)
        nn = np.linalg.norm(un)
        if nn > 1e-14 * max(np.linalg.norm(u), 1e-300):
            return np.concatenate([Vt, (un / nn)[:, None]], 1)
        return Vt

    # -- Alg. "UPDATE-PARAM" (per view) ---------------------------------------
    def view_terms(self, theta, u):
        """Per view: gradient g_v, |J_v|^2, misfit f_v and the rounding scale
        rho_v = sum_b |r_b| (|(H u)_b| + |b_b|) of f_v."""
        g = self.g
        Hu = self.H(theta, u).reshape(g.V, g.B)
        bv = self.b.reshape(g.V, g.B)
        r = Hu - bv
        dt, _ = dsample(g, theta, u, self.delta)
        dt = dt.reshape(g.V, g.B)
        rho = (np.abs(r) * (np.abs(Hu) + np.abs(bv))).sum(1)
        return (r * dt).sum(1), (dt * dt).sum(1), 0.5 * (r * r).sum(1), rho

    def view_f(self, theta, u):
        g = self.g
        r = (self.H(theta, u) - self.b).reshape(g.V, g.B)
        return 0.5 * (r * r).sum(1)

    def update_param(self, theta, u):
        o = self.o
        theta = theta.copy()
        for _ in range(o.maxiter_p):
            grad, jn2, f0, rho = self.view_terms(theta, u)
            mu = o.mu_rel * max(float(jn2.max()), 1e-300)
            d = -grad / (jn2 + mu)
            alpha = np.full(theta.shape, o.alpha0)
            active = np.ones(theta.shape, bool)
            trials = np.zeros(theta.shape, int)
            for _h in range(o.max_halvings + 1):
                # noise floor: the first-order change of f_v is below its rounding
                low = active & (alpha * np.abs(grad * d) < o.armijo_eps * rho)
                alpha[low] = 0.0
                active &= ~low
                if not active.any():
                    break
                ft = self.view_f(theta + alpha * d, u)
                trials += active
                ok = ft <= f0 + o.c1 * alpha * grad * d
                active &= ~ok
                if not active.any():
                    break
                alpha[active] *= o.beta
            alpha[active] = 0.0  # no acceptable step for these views
            theta = theta + alpha * d
            self.last_trials = trials
        return theta

    def update_param_shared(self, theta, u):
        """UPDATE-PARAM for one offset p shared by every view: theta + p 1."""
        o = self.o
        theta = theta.copy()
        for _ in range(o.maxiter_p):
            grad, jn2, f0, rho = self.view_terms(theta, u)
            g, jj, f, r = float(grad.sum()), float(jn2.sum()), float(f0.sum()), float(rho.sum())
            d = -g / (jj + o.mu_rel * max(jj, 1e-300))
            alpha = o.alpha0
            accepted = False
            self.last_trials = 0
            for _h in range(o.max_halvings + 1):
                if alpha * abs(g * d) < o.armijo_eps * r:
                    break  # noise floor: the first-order change of f is below its rounding
                ft = float(self.view_f(theta + alpha * d, u).sum())
                self.last_trials += 1
                if ft <= f + o.c1 * alpha * g * d:
                    accepted = True
                    break
                alpha *= o.beta
            if not accepted:
                break  # no acceptable step: the offset stays
            theta = theta + alpha * d
        return theta

    # -- Alg. "UPDATE-PARAM-VarPro" (Sec. 4.2) ----------------------------------
    def update_param_varpro(self, theta, V, lam, w):
        """maxiter_p Gauss-Newton steps on the reduced objective f(theta) on the
        basis V with frozen weights w (P^2) and lambda_hat = lam."""
        o, g = self.o, self.g
        theta = np.array(theta, float)
        for _ in range(o.maxiter_p):
            Jr, Js, r, s, f0, u = varpro_jacobians(g, self.b, theta, V, lam, w, self.delta, o.temporal)
            rho = float(np.sum(np.abs(r) * (np.abs(r + self.b) + np.abs(self.b))))
            # gradient of J_{eps,lambda}(u_hat, theta) in theta: only the data term depends on theta
            grad, _ = jacT(g, theta, u, r, self.delta)
            A = Jr.T @ Jr + lam * (Js.T @ Js)
            mu = o.mu_rel * max(float(np.max(np.diag(A))), 1e-300)
            d = -np.linalg.solve(A + mu * np.eye(g.V), grad)
            gd = float(grad @ d)
            alpha = o.alpha0
            accepted = False
            self.last_trials = 0
            for _h in range(o.max_halvings + 1):
                if alpha * abs(gd) < o.armijo_eps * rho:
                    break  # noise floor: the first-order change of f is below its rounding
                ft = varpro_objective(g, self.b, theta + alpha * d, V, lam, w, self.delta, o.temporal)[0]
                self.last_trials += 1
                if ft <= f0 + o.c1 * alpha * gd:
                    accepted = True
                    break
                alpha *= o.beta
            if not accepted:
                break  # no acceptable step: the angles stay
            theta = theta + alpha * d
        return theta

    def param_update(self, theta, u, V, lam):
        """UPDATE-PARAM of the outer iteration: per-view AltMin, or VarPro on
        the compressed basis V with the MM weights of u."""
        if self.o.shared_offset:
            if self.o.varpro:
                raise ValueError("the shared offset is updated by UPDATE-PARAM, not the VarPro update")
            return self.update_param_shared(theta, u)
        if not self.o.varpro:
            return self.update_param(theta, u)
        o = self.o
        w = o.fixed_weights if o.fixed_weights is not None else mm_weights(psi(self.g, u, o.temporal), o.eps)
        return self.update_param_varpro(theta, V, lam, w)

    # -- residual of the normal equations appended to V -----------------------
    def residual_direction(self, theta, u, lam, V):
        g = self.g
        tm = self.o.temporal
        w = self.o.fixed_weights if self.o.fixed_weights is not None else mm_weights(psi(g, u, tm), self.o.eps)
        r = self.HT(theta, self.H(theta, u) - self.b) + lam * psi_t(g, w * psi(g, u, tm), tm)
        r = cgs2(V, r)
        nr = np.linalg.norm(r)
        return r / nr if nr > 0 else None

    # -- Alg. "NL-RMM-GKS" -------------------------------------------------------
    def solve(self, theta0, u_true=None, theta_true=None, callback=None):
        o, g = self.o, self.g
        theta = np.array(theta0, float)
        u = np.zeros(g.n)
        V = self.gkb(theta, o.k_min)
        hist = History()
        s = o.k_max - o.k_min
        lam = None
        for it in range(o.outer_iters):
            HV = np.stack([self.H(theta, V[:, j]) for j in range(V.shape[1])], 1)
            u_new, lam, Vg, _, RH, RP, used, steps = self.enlarge(theta, V, HV, u, s)
            Vk = self.compress(Vg, RH, RP, used, lam, u_new)
            theta_new = self.param_update(theta, u_new, Vk, lam) if o.update_theta else theta.copy()
            vn = self.residual_direction(theta, u_new, lam, Vk)
            V = Vk if vn is None else np.concatenate([Vk, vn[:, None]], 1)
            nu = np.linalg.norm(u)
            du = np.linalg.norm(u_new - u) / nu if nu > 0 else np.inf
            dth = float(np.linalg.norm(theta_new - theta))
            hist.lam.append(lam)
            hist.du.append(du)
            hist.dtheta.append(dth)
            hist.enlarge_steps.append(steps)
            if u_true is not None:
                hist.rre.append(float(np.linalg.norm(u_new - u_true) / np.linalg.norm(u_true)))
            if theta_true is not None:
                hist.angle_err.append(float(np.linalg.norm(theta_new - theta_true) / np.linalg.norm(theta_true)))
            u, theta = u_new, theta_new
            if callback:
                callback(it, u, theta, V, lam)
            if o.stop_on_convergence and du < o.tol_u and dth < o.tol_p:
                break
        return u, theta, hist


# ---------------------------------------------------------------------------
# VarPro reduced objective on a fixed basis (Sec. 4.2, Alg. "UPDATE-PARAM-VarPro")
# ---------------------------------------------------------------------------
def varpro_objective(g: Geometry, b, theta, V, lam, w=None, delta=None, temporal=False):
    """f(theta) = min_y 1/2 |H(theta) V y - b|^2 + lam/2 |P Psi V y|^2 with P^2 = diag(w)
    (w = None: P = I), solved through the QR factors of H V and P Psi V as in the
    reduced problem (3.5).  Returns (f, y, u = V y)."""
    HV = np.stack([forward(g, theta, V[:, j], delta) for j in range(V.shape[1])], 1)
    PsiV = np.stack([psi(g, V[:, j], temporal) for j in range(V.shape[1])], 1)
    if w is not None:
        PsiV = np.sqrt(w)[:, None] * PsiV
    QH, RH = np.linalg.qr(HV)
    _, RP = np.linalg.qr(PsiV)
    y = np.linalg.solve(RH.T @ RH + lam * (RP.T @ RP), RH.T @ (QH.T @ b))
    r = HV @ y - b
    s = PsiV @ y
    return 0.5 * r @ r + 0.5 * lam * s @ s, y, V @ y


def varpro_gradient(g: Geometry, b, theta, V, lam, w=None, delta=None, temporal=False):
    """grad_theta f: y is optimal for every theta, so by the Golub-Pereyra
    (envelope) argument the reduced gradient is J_theta(u)^T (H(theta) u - b)
    with u = V y(theta), the data-term gradient (H_{p_i} u)^T (H u - b)."""
    f, y, u = varpro_objective(g, b, theta, V, lam, w, delta, temporal)
    r = forward(g, theta, u, delta) - b
    gt, _ = jacT(g, theta, u, r, delta)
    return gt, f, u


def varpro_jacobians(g: Geometry, b, theta, V, lam, w=None, delta=None, temporal=False):
    """Jacobians of the reduced residuals r(theta) = H(theta) V y(theta) - b and
    s(theta) = P Psi V y(theta) of f = 1/2 |r|^2 + lam/2 |s|^2 (Sec. 4.2).

    Column j (angle of view j) follows the sensitivity equation restricted to
    span(V) (u_{p_j} = V y_j):
        M y_j = -((H_j V)^T r + (H V)^T H_j u),  M = (HV)^T HV + lam (P Psi V)^T (P Psi V),
        J_r[:, j] = H_j u + (H V) y_j,           J_s[:, j] = (P Psi V) y_j,
    with H_j = dH/dtheta_j applied through the oracle's Jacobian (direction e_j).
    One column at a time, dense.  Returns (J_r, J_s, r, s, f, u)."""
    k = V.shape[1]
    f, y, u = varpro_objective(g, b, theta, V, lam, w, delta, temporal)
    HV = np.stack([forward(g, theta, V[:, c], delta) for c in range(k)], 1)
    PsiV = np.stack([psi(g, V[:, c], temporal) for c in range(k)], 1)
    if w is not None:
        PsiV = np.sqrt(w)[:, None] * PsiV
    r = HV @ y - b
    s = PsiV @ y
    M = HV.T @ HV + lam * (PsiV.T @ PsiV)
    Jr = np.empty((r.size, g.V))
    Js = np.empty((s.size, g.V))
    for j in range(g.V):
        e = np.zeros(g.V)
        e[j] = 1.0
        Hju = jac(g, theta, u, e, delta)
        HjV = np.stack([jac(g, theta, V[:, c], e, delta) for c in range(k)], 1)
        yj = -np.linalg.solve(M, HjV.T @ r + HV.T @ Hju)
        Jr[:, j] = Hju + HV @ yj
        Js[:, j] = PsiV @ yj
    return Jr, Js, r, s, f, u


# ---------------------------------------------------------------------------
# Alg. "s-NL-RMM-GKS" (Sec. 5): streaming over measurement blocks
# ---------------------------------------------------------------------------
def stream_solve(blocks, theta0, passes, u_true=None, theta_true=None, tol_u=None, tol_p=None, callback=None):
    """Streaming NL-RMM-GKS over blocks of views (Sec. 2.4 block setup, Sec. 5).

    ``blocks``: one NLRMMGKS per block j (its views' geometry, b_j, options
    with that block's noise norm); all share the image size.  ``theta0``: the
    blocks' initial angles.  Each pass visits the blocks in order; a visit is
    one RMM-GKS cycle (Enlarge + Compress) on block j's data started from the
    carried image and compressed basis, then UPDATE-PARAM for block j's
    angles; the compressed basis is carried to the next block.  After each
    pass the change of u and of all angles over the pass is checked against
    tol_u / tol_p (the options of block 1 when not given).

    Readings: V^(0)_kmin is the GKB basis of block 1 (b_1, k_min steps); no
    residual is appended after the parameter update (the printed algorithm
    has none: the first Enlarge step of the next block appends that block's
    residual); the optional high-lambda solve is off.
    Returns (u, thetas, history) with one history entry per pass;
    ``callback(pass, j, u, V, thetas)`` after each block visit.
    """
    o1 = blocks[0].o
    tol_u = o1.tol_u if tol_u is None else tol_u
    tol_p = o1.tol_p if tol_p is None else tol_p
    thetas = [np.array(t, float) for t in theta0]
    n = blocks[0].g.n
    u = np.zeros(n)
    V = blocks[0].gkb(thetas[0], o1.k_min)
    hist = History()
    for _ in range(passes):
        u_start = u.copy()
        th_start = [t.copy() for t in thetas]
        steps_pass = 0
        lam = None
        for j, blk in enumerate(blocks):
            th = thetas[j]
            HV = np.stack([blk.H(th, V[:, c]) for c in range(V.shape[1])], 1)
            u, lam, Vg, _, RH, RP, used, steps = blk.enlarge(th, V, HV, u, blk.o.k_max - blk.o.k_min)
            V = blk.compress(Vg, RH, RP, used, lam, u)
            thetas[j] = blk.param_update(th, u, V, lam) if blk.o.update_theta else th.copy()
            steps_pass += steps
            if callback:
                callback(len(hist.du), j, u, V, thetas)
        nu = np.linalg.norm(u_start)
        du = np.linalg.norm(u - u_start) / nu if nu > 0 else np.inf
        dth = float(np.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(thetas, th_start))))
        hist.lam.append(lam)
        hist.du.append(du)
        hist.dtheta.append(dth)
        hist.enlarge_steps.append(steps_pass)
        if u_true is not None:
            hist.rre.append(float(np.linalg.norm(u - u_true) / np.linalg.norm(u_true)))
        if theta_true is not None:
            err = np.concatenate([a - b for a, b in zip(thetas, theta_true)])
            hist.angle_err.append(float(np.linalg.norm(err) / np.linalg.norm(np.concatenate(theta_true))))
        if o1.stop_on_convergence and du < tol_u and dth < tol_p:
            break
    return u, thetas, hist
