"""Band-staged FP32 ray march against the L1-gather march and the oracle.

The staged kernels sum every ray row by row in increasing row order with the
same fused multiply-adds as the L1-gather kernels with one row segment per
ray, so forward, JVP, VJP and the Gauss-Newton terms must agree bit for bit,
whether a row block is read from shared memory or (band wider than the
buffer, or views of one CTA on different frames or axes) from global memory.
With several CTAs per ray (row segments) the staged forward must equal the
L1-gather forward with the same number of row segments per ray.  The cases
cover an odd image side (odd pair pitch: 8-byte copies), uneven
frames with an empty one, axis-aligned views (every row marched), ragged
batches and chunks, and sparse angle sets whose bands overflow the buffer.
"""
import numpy as np
import pytest

import oracle
from paper_2605_06336_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.double().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _angles(kind, V, rng):
    if kind == "random":
        return synth.random_angles(V, rng)
    if kind == "sparse":  # few views over [0, pi): neighbouring views far apart, wide bands
        return np.sort(rng.uniform(0, np.pi, V))
    # near the axes: exact 0, pi/2 + 1e-7, and small slopes that march every row
    th = synth.random_angles(V, rng)
    th[0] = 0.0
    th[1 % V] = np.pi / 2 + 1e-7
    th[2 % V] = 1e-3
    th[3 % V] = np.pi - 2e-3
    return th


CASES = [
    # N, views per frame, batch, angle kind
    (256, [180], 8, "random"),
    (37, [11, 0, 6], 3, "axes"),
    (64, [30, 17], 5, "random"),
    (129, [40], 2, "axes"),
    (512, [16], 1, "sparse"),
]
SHAPES = [(4, 4, 1), (8, 8, 2), (4, 8, 4), (8, 4, 1), (8, 4, 2)]  # (views per CTA, rows per block, CTAs per ray)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{c[0]}_F{len(c[1])}_K{c[2]}_{c[3]}")
def test_band_matches_gather_bit_for_bit(case):
    from paper_2605_06336_gb300 import ct
    N, vpf, K, kind = case
    B = synth.n_bins(N)
    V = sum(vpf)
    rng = np.random.default_rng(N + K)
    theta = _angles(kind, V, rng)
    delta = rng.normal(0, 0.5, V)
    X = rng.uniform(size=(K, len(vpf) * N * N))
    R = rng.standard_normal(V * B)
    dth = rng.standard_normal(V)
    ddl = rng.standard_normal(V)
    op = ct.CTOperator(N, B, V, vpf, max_batch=K, dtype=torch.float32)
    th, dl = dev(theta), dev(delta)
    Xg, Rg = dev(X, torch.float32), dev(R, torch.float32)
    kb = 8 if K >= 8 else (4 if K >= 4 else (2 if K >= 2 else 1))

    def run(tuning):
        op.tuning = tuning
        y = op.forward(Xg, th, dl).clone()
        j = op.jac(Xg[0], th, dev(dth), dl, dev(ddl)).clone()
        gt, gd = op.jacT(Xg[0], th, Rg, dl, want_delta=True)
        g, j2, f, res = op.gn_terms(Xg[0], th, Rg, dl, want_residual=True)
        return [y, j, gt.clone(), gd.clone(), g.clone(), j2.clone(), f.clone(), res.clone()]

    for vw, rb, segs in SHAPES:
        # L1-gather reference: the same row segments per ray (as warps of one CTA), whole rays for J
        ref = run([kb, segs, 1, 1, 1, 1, 1, 0, 0, 0, 1])
        got = run([kb, segs, vw, 1, 1, 1, vw, rb, rb, 0, 1])
        for name, a, b in zip(("forward", "jvp", "vjp_theta", "vjp_delta", "gn_grad", "gn_j2", "gn_f", "gn_res"),
                              got, ref):
            assert torch.equal(a, b), (name, vw, rb, segs, float((a.double() - b.double()).abs().max()))
    g_o = oracle.Geometry(N, B, V, vpf)
    assert rel(host(got[0]), oracle.forward(g_o, theta, X, delta)) <= 1e-5
    assert rel(host(got[1]), oracle.jac(g_o, theta, X[0], dth, delta, ddl)) <= 1e-5


def test_band_forward_full_batch_matches_oracle():
    """The headline 256^2 / 180-view / 8-image block through the staged forward, against the oracle."""
    from paper_2605_06336_gb300 import ct
    w = synth.make_workload("C2")
    K = 8
    rng = np.random.default_rng(3)
    X = np.concatenate([w.images.reshape(1, -1), rng.uniform(size=(K - 1, w.N * w.N))])
    op = ct.CTOperator(w.N, w.B, w.V, max_batch=K, dtype=torch.float32)
    op.tuning = [8, 2, 8, 8, 2, 1, 8, 4, 4, 0, 1]
    y = host(op.forward(dev(X, torch.float32), dev(w.theta_true)))
    g = oracle.Geometry(w.N, w.B, w.V)
    assert rel(y, oracle.forward(g, w.theta_true, X)) <= 1e-5


ADJ_SHAPES = [(8, 1), (16, 2), (8, 4), (16, 1)]  # (views per staged block, CTAs per tile)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{c[0]}_F{len(c[1])}_K{c[2]}_{c[3]}")
def test_staged_transpose_matches_gather_bit_for_bit(case):
    """The staged transpose sums each pixel's views in the order of k_adjoint
    with the same number of view groups, so the two agree bit for bit."""
    from paper_2605_06336_gb300 import ct
    N, vpf, K, kind = case
    B = synth.n_bins(N)
    V = sum(vpf)
    rng = np.random.default_rng(3 * N + K)
    theta = _angles(kind, V, rng)
    delta = rng.normal(0, 0.5, V)
    Y = rng.standard_normal((K, V * B))
    op = ct.CTOperator(N, B, V, vpf, max_batch=K, dtype=torch.float32)
    th, dl, Yg = dev(theta), dev(delta), dev(Y, torch.float32)
    for akb in sorted({1, 2, 4, 8} & set(range(1, K + 1))):
        for vb, segs in ADJ_SHAPES:
            op.tuning = [1, 1, 1, akb, segs, 1, 1, 0, 0, 0, 1]
            ref = op.adjoint(Yg, th, dl).clone()
            op.tuning = [1, 1, 1, akb, segs, 1, 1, 0, 0, vb, 1]
            got = op.adjoint(Yg, th, dl).clone()
            assert torch.equal(got, ref), (akb, vb, segs, float((got - ref).abs().max()))
    g_o = oracle.Geometry(N, B, V, vpf)
    assert rel(host(got), oracle.adjoint(g_o, theta, Y, delta)) <= 1e-5
