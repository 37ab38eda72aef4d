"""The autograd Function: gradients against the oracle and against central differences.

Loss L = <w, H(theta, delta) x> for a fixed random w: dL/dx = H^T w,
dL/dtheta = J_theta^T w, dL/ddelta = J_delta^T w (oracle), and the
directional derivatives along 32 random directions match central differences
of the FP64 GPU forward: interpolation kinks crossed inside [-h, h] make the
quotient O(h)-accurate, so the error must shrink linearly from h = 1e-4 to
h = 1e-6 (the same property the oracle's own pin checks).
"""
import numpy as np
import pytest

import oracle
from paper_2605_06336_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(scale=0.25, dtype=torch.float32):
    from paper_2605_06336_gb300 import ct
    w = synth.make_workload("C3", scale=scale)  # 512^2 / 360 views / offsets, scaled down
    op = ct.CTOperator(w.N, w.B, w.V, max_batch=2, dtype=dtype)
    return w, op


def test_gradients_match_the_oracle():
    from paper_2605_06336_gb300.autograd import project
    w, op = _setup()
    rng = np.random.default_rng(1)
    x_np = np.stack([w.images.reshape(-1), rng.uniform(size=w.N * w.N)])
    wt_np = rng.standard_normal((2, w.V * w.B))
    x = torch.tensor(x_np, dtype=torch.float32, device="cuda", requires_grad=True)
    th = torch.tensor(w.theta_true, dtype=torch.float64, device="cuda", requires_grad=True)
    dl = torch.tensor(w.delta_true, dtype=torch.float64, device="cuda", requires_grad=True)
    wt = torch.tensor(wt_np, dtype=torch.float32, device="cuda")
    y = project(x, th, op, dl)
    loss = (y.double() * wt.double()).sum()
    loss.backward()
    g = oracle.Geometry(w.N, w.B, w.V)
    gx_o = oracle.adjoint(g, w.theta_true, wt_np, w.delta_true)
    gt_o = np.zeros(w.V)
    gd_o = np.zeros(w.V)
    for k in range(2):
        a, b = oracle.jacT(g, w.theta_true, x_np[k], wt_np[k], w.delta_true)
        gt_o += a
        gd_o += b
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(x.grad.double().cpu().numpy(), gx_o) <= 1e-5
    assert rel(th.grad.cpu().numpy(), gt_o) <= 1e-5
    assert rel(dl.grad.cpu().numpy(), gd_o) <= 1e-5


def test_directional_derivatives_match_central_differences():
    from paper_2605_06336_gb300.autograd import project
    w, op = _setup(dtype=torch.float64)
    rng = np.random.default_rng(2)
    x = torch.tensor(w.images.reshape(-1), dtype=torch.float64, device="cuda")
    th0 = torch.tensor(w.theta_true, dtype=torch.float64, device="cuda")
    dl0 = torch.tensor(w.delta_true, dtype=torch.float64, device="cuda")
    wt = torch.tensor(rng.standard_normal(w.V * w.B), dtype=torch.float64, device="cuda")
    th = th0.clone().requires_grad_(True)
    dl = dl0.clone().requires_grad_(True)
    (project(x, th, op, dl) * wt).sum().backward()
    dirs = [(torch.tensor(rng.standard_normal(w.V), dtype=torch.float64, device="cuda"),
             torch.tensor(rng.standard_normal(w.V), dtype=torch.float64, device="cuda")) for _ in range(32)]
    errs = {}
    for h in (1e-4, 1e-5, 1e-6):
        err = ref = 0.0
        for dth, ddl in dirs:
            lp = float((op.forward(x, th0 + h * dth, dl0 + h * ddl) * wt).sum())
            lm = float((op.forward(x, th0 - h * dth, dl0 - h * ddl) * wt).sum())
            fd = (lp - lm) / (2 * h)
            an = float((th.grad * dth).sum() + (dl.grad * ddl).sum())
            err += abs(fd - an)
            ref += abs(an)
        errs[h] = err / ref
    assert errs[1e-4] <= 5e-2, errs
    assert errs[1e-6] <= errs[1e-4] / 20, errs
    assert errs[1e-6] <= 1e-3, errs
