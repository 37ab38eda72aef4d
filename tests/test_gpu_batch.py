"""Batched Jacobian products (ct_jac_batch, ct_jacT_batch, ct_gn_terms_batch) through the C ABI.

K images sharing the angles go through one ray-march launch (the basis block of
Sec. 3.2, whose sensitivities enter the VarPro Gauss-Newton system of Sec. 4.2).
* every image's result equals the FP64 oracle's on that image within the
  operator tolerances (1e-5 float32, 1e-12 float64; normwise and per view),
  for K = 1, 3, 8, 11 (groups of 4 + 4 + 2 + 1 images per lane), frames with
  uneven view counts (one empty), offsets, per-image and shared directions,
  per-image and shared residuals, and the sum over the images;
* every image's result is bit-identical to the single-image call on it at
  1, 2 and 4 images per lane: batching shares the line, cell and fraction of
  a ray between images and leaves each image's summation order unchanged;
* the fan-beam handle batches its angle and offset derivatives the same way.
"""
import numpy as np
import pytest

import oracle
from paper_2605_06336_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float32: 1e-5, torch.float64: 1e-12}


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def view_sum_rel(gv, go, r, dt, V, B):
    mag = (np.abs(np.asarray(r).reshape(V, B)) * np.abs(np.asarray(dt).reshape(V, B))).sum(1)
    mag[mag == 0] = 1.0
    return float((np.abs(np.asarray(gv) - np.asarray(go)) / mag).max()) if V else 0.0


def _problem(N, vpf, K, offs, seed):
    rng = np.random.default_rng(seed)
    V = sum(vpf)
    B = synth.n_bins(N)
    theta = synth.random_angles(V, rng)
    delta = rng.normal(0, 0.5, V) if offs else None
    X = rng.uniform(size=(K, len(vpf) * N * N))
    R = rng.standard_normal((K, V * B))
    D = rng.standard_normal((K, V))
    DD = rng.standard_normal((K, V)) if offs else None
    return oracle.Geometry(N, B, V, vpf), theta, delta, X, R, D, DD


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("K,N,vpf,offs", [(1, 24, [13], True), (3, 37, [11], False), (8, 32, [5, 0, 9, 4], True),
                                          (11, 29, [17], False)])
def test_batched_products_match_the_oracle(K, N, vpf, offs, dtype):
    from paper_2605_06336_gb300 import ct
    g, theta, delta, X, R, D, DD = _problem(N, vpf, K, offs, seed=100 + K)
    V, B = g.V, g.B
    op = ct.CTOperator(N, B, V, vpf, max_batch=K, dtype=dtype)
    th, dl = dev(theta), (dev(delta) if offs else None)
    Xg, Rg = dev(X, dtype), dev(R, dtype)
    dY = host(op.jac_batch(Xg, th, dev(D), dl, dev(DD) if offs else None))          # per-image directions
    dY1 = host(op.jac_batch(Xg, th, dev(D[0]), dl, dev(DD[0]) if offs else None))   # one shared direction
    out = op.jacT_batch(Xg, th, Rg, dl, want_delta=offs)
    gt, gd = (out if offs else (out, None))
    gt_shared = host(op.jacT_batch(Xg, th, Rg[0], dl))
    gt_sum = host(op.jacT_batch(Xg, th, Rg, dl, sum_images=True))
    gr, j2, f, res = op.gn_terms_batch(Xg, th, Rg, dl, want_residual=True)
    torch.cuda.synchronize()
    tol = TOL[dtype]
    gsum_o = np.zeros(V)
    for k in range(K):
        dyo = oracle.jac(g, theta, X[k], D[k], delta, DD[k] if offs else None)
        assert rel(dY[k], dyo) <= tol
        assert rel(dY1[k], oracle.jac(g, theta, X[k], D[0], delta, DD[0] if offs else None)) <= tol
        dt, dd = oracle.dsample(g, theta, X[k], delta)
        gto, gdo = oracle.jacT(g, theta, X[k], R[k], delta)
        assert view_sum_rel(host(gt[k]), gto, R[k], dt, V, B) <= tol
        if offs:
            assert view_sum_rel(host(gd[k]), gdo, R[k], dd, V, B) <= tol
        gto0, _ = oracle.jacT(g, theta, X[k], R[0], delta)
        assert view_sum_rel(gt_shared[k], gto0, R[0], dt, V, B) <= tol
        gsum_o += gto
        r_o = oracle.forward(g, theta, X[k], delta) - R[k]
        assert rel(host(res[k]), r_o) <= tol
        Rk, dtk = r_o.reshape(V, B), dt.reshape(V, B)
        assert view_sum_rel(host(gr[k]), (Rk * dtk).sum(1), Rk, dtk, V, B) <= tol
        if V:
            assert np.max(np.abs(host(j2[k]) / np.maximum((dtk * dtk).sum(1), 1e-300) - 1)) <= tol
            assert np.max(np.abs(host(f[k]) / (0.5 * (Rk * Rk).sum(1)) - 1)) <= tol
    if V:
        mag = sum((np.abs(R[k].reshape(V, B)) * np.abs(oracle.dsample(g, theta, X[k], delta)[0].reshape(V, B))).sum(1)
                  for k in range(K))
        assert float(np.max(np.abs(gt_sum - gsum_o) / mag)) <= tol


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("kb", [1, 2, 4])
def test_batched_products_equal_the_single_image_calls_bit_for_bit(kb, dtype):
    from paper_2605_06336_gb300 import ct
    K, N, vpf = 7, 48, [20, 17]
    g, theta, delta, X, R, D, DD = _problem(N, vpf, K, True, seed=7)
    op = ct.CTOperator(N, g.B, g.V, vpf, max_batch=K, dtype=dtype)
    t = op.tuning
    t[10] = kb
    op.tuning = t
    th, dl = dev(theta), dev(delta)
    Xg, Rg = dev(X, dtype), dev(R, dtype)
    dY = op.jac_batch(Xg, th, dev(D), dl, dev(DD))
    gt, gd = op.jacT_batch(Xg, th, Rg, dl, want_delta=True)
    gsum = op.jacT_batch(Xg, th, Rg, sum_images=True)
    gr, j2, f, res = op.gn_terms_batch(Xg, th, Rg, dl, want_residual=True)
    for k in range(K):
        assert torch.equal(dY[k], op.jac(Xg[k], th, dev(D[k]), dl, dev(DD[k])))
        a, b = op.jacT(Xg[k], th, Rg[k], dl, want_delta=True)
        assert torch.equal(gt[k], a) and torch.equal(gd[k], b)
        g1, j1, f1, r1 = op.gn_terms(Xg[k], th, Rg[k], dl, want_residual=True)
        assert torch.equal(gr[k], g1) and torch.equal(j2[k], j1) and torch.equal(f[k], f1)
        assert torch.equal(res[k], r1)
    # the sum over images adds the per-image sums in image order (0 + s_0 + s_1 + ...)
    acc = torch.zeros(g.V, dtype=torch.float64, device="cuda")
    for k in range(K):
        acc = acc + op.jacT(Xg[k], th, Rg[k])
    assert torch.equal(gsum, acc)


def test_fan_beam_batched_angle_derivatives():
    from paper_2605_06336_gb300 import ct
    K, N, V = 5, 32, 24
    rng = np.random.default_rng(9)
    B, D = synth.n_bins(N), 64.0
    g = oracle.Geometry(N, B, V, fan_D=D)
    theta = synth.random_angles(V, rng)
    X = rng.uniform(size=(K, N * N))
    R = rng.standard_normal((K, V * B))
    dth = rng.standard_normal(V)
    op = ct.CTOperator(N, B, V, max_batch=K, dtype=torch.float32, source_distance=D)
    th = dev(theta)
    dY = host(op.jac_batch(dev(X, torch.float32), th, dev(dth)))
    gt = host(op.jacT_batch(dev(X, torch.float32), th, dev(R, torch.float32)))
    for k in range(K):
        assert rel(dY[k], oracle.jac(g, theta, X[k], dth)) <= 1e-5
        assert rel(gt[k], oracle.jacT(g, theta, X[k], R[k])[0]) <= 1e-5
    # with offsets: J_theta dtheta + J_delta ddelta and both gradients per image
    delta = rng.normal(0, 0.5, V)
    ddl = rng.standard_normal(V)
    dY = host(op.jac_batch(dev(X, torch.float32), th, dev(dth), dev(delta), dev(ddl)))
    gt, gd = op.jacT_batch(dev(X, torch.float32), th, dev(R, torch.float32), dev(delta), want_delta=True)
    for k in range(K):
        assert rel(dY[k], oracle.jac(g, theta, X[k], dth, delta, ddl)) <= 1e-5
        a, b = oracle.jacT(g, theta, X[k], R[k], delta)
        assert rel(host(gt[k]), a) <= 1e-5 and rel(host(gd[k]), b) <= 1e-5


def test_batched_argument_errors():
    from paper_2605_06336_gb300 import ct
    op = ct.CTOperator(16, 23, 6, max_batch=2, dtype=torch.float32)
    lib = ct.load_library()
    X = torch.zeros(3, 256, device="cuda")
    th = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        op.jac_batch(X, th, th)                 # batch above max_batch
    p = ctypes_ptr = X.data_ptr()
    assert lib.ct_jac_batch(op.h, th.data_ptr(), None, p, th.data_ptr(), None, p, 3, 0) == ct.CT_ERR_ARG
    assert lib.ct_jac_batch(op.h, th.data_ptr(), None, p, th.data_ptr(), None, p, 1, 8) == ct.CT_ERR_ARG
    assert lib.ct_jacT_batch(op.h, th.data_ptr(), None, p, p, th.data_ptr(), None, 0, 0) == ct.CT_ERR_ARG
    assert lib.ct_jacT_batch(op.h, th.data_ptr(), None, p, p, th.data_ptr(), None, 1, 1) == ct.CT_ERR_ARG
    assert lib.ct_gn_terms_batch(op.h, th.data_ptr(), None, p, p, None, th.data_ptr(), th.data_ptr(), None,
                                 5) == ct.CT_ERR_ARG
    del ctypes_ptr
