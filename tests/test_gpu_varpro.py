"""VarPro reduced objective and gradient on the GPU (nlrmm_varpro, autograd) against the oracle.

f(theta) = min_y 1/2 |H(theta) V y - b|^2 + lam/2 |P Psi V y|^2 on a fixed basis V
with frozen MM weights; grad f = J_theta(V y)^T (H V y - b).  The autograd
Function recomputes the reduced solve in backward (nothing stored).
"""
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
    assert rel(grad.cpu().numpy(), gt_o) <= tol * 10


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
