"""Batched frames and Krylov block in one persistent launch, captured in a CUDA graph.

The operator step (H on a Krylov block of 8 dynamic images, H^T on 8 sinograms,
J dtheta, J^T r) over 16 frames with uneven view counts is captured once and
replayed on new inputs; every replay must reproduce the eager launches bit
for bit (the kernels reduce in a fixed order) and match the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2605_06336_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_graph_replay_matches_eager_and_oracle():
    from paper_2605_06336_gb300 import ct
    w = synth.make_workload("C4", scale=0.25)     # 16 frames of 64^2, 7..30 golden-angle views each
    N, B, V, F, K = w.N, w.B, w.V, w.F, 8
    op = ct.CTOperator(N, B, V, w.views_per_frame, max_batch=K, dtype=torch.float32)
    op.autotune()
    n, m = op.n, op.m
    rng = np.random.default_rng(5)
    th = torch.tensor(w.theta_true, dtype=torch.float64, device="cuda")
    dth = torch.tensor(rng.standard_normal(V), dtype=torch.float64, device="cuda")
    X = torch.zeros(K, n, device="cuda")
    Ys = torch.zeros(K, m, device="cuda")
    Y = torch.empty(K, m, device="cuda")
    Xa = torch.empty(K, n, device="cuda")
    dy = torch.empty(m, device="cuda")
    gt = torch.empty(V, dtype=torch.float64, device="cuda")

    def step():
        ct.ct_forward(op.h, th, None, X, Y, K)
        ct.ct_adjoint(op.h, th, None, Ys, Xa, K)
        ct.ct_jac(op.h, th, None, X[0], dth, None, dy)
        ct.ct_jacT(op.h, th, None, X[0], Ys[0], gt, None)

    def fill(seed):
        r = np.random.default_rng(seed)
        X.copy_(torch.tensor(r.uniform(size=(K, n)), dtype=torch.float32))
        Ys.copy_(torch.tensor(r.standard_normal((K, m)), dtype=torch.float32))

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        op.set_stream(side)
        fill(1)
        step()  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        op.set_stream(torch.cuda.current_stream())
        step()
    op.set_stream(torch.cuda.current_stream())
    for seed in (2, 3):
        fill(seed)
        g.replay()
        torch.cuda.synchronize()
        got = [t.clone() for t in (Y, Xa, dy, gt)]
        step()                                        # eager, same inputs
        torch.cuda.synchronize()
        for a, b in zip(got, (Y, Xa, dy, gt)):
            assert torch.equal(a, b)
    g_o = oracle.Geometry(N, B, V, w.views_per_frame)
    Xh = X.double().cpu().numpy()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(Y.double().cpu().numpy(), oracle.forward(g_o, w.theta_true, Xh)) <= 1e-5
    assert rel(Xa.double().cpu().numpy(), oracle.adjoint(g_o, w.theta_true, Ys.double().cpu().numpy())) <= 1e-5


def test_two_handles_on_two_streams_in_one_graph():
    """The bench's overlapped step: H^T on a second handle of the same geometry,
    on its own stream, forked from and joined back into the capturing stream
    (a parallel branch of one CUDA graph), while H, J and J^T run on the first
    handle.  Handles share no workspace, so the replay gives, bit for bit, what
    the four calls in order on one handle give."""
    from paper_2605_06336_gb300 import ct
    w = synth.make_workload("C2", scale=0.25)
    N, B, V, K = w.N, w.B, w.V, 8
    op = ct.CTOperator(N, B, V, max_batch=K, dtype=torch.float32)
    opT = ct.CTOperator(N, B, V, max_batch=K, dtype=torch.float32)
    opT.tuning = op.tuning
    rng = np.random.default_rng(9)
    th = torch.tensor(w.theta_true, dtype=torch.float64, device="cuda")
    dth = torch.tensor(rng.standard_normal(V), dtype=torch.float64, device="cuda")
    X = torch.tensor(rng.uniform(size=(K, op.n)), dtype=torch.float32, device="cuda")
    Ys = torch.tensor(rng.standard_normal((K, op.m)), dtype=torch.float32, device="cuda")
    Y, Xa = torch.empty(K, op.m, device="cuda"), torch.empty(K, op.n, device="cuda")
    dy, gt = torch.empty(op.m, device="cuda"), torch.empty(V, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()

    def overlapped():
        cur = torch.cuda.current_stream()
        fork = torch.cuda.Event()
        fork.record(cur)
        side.wait_event(fork)
        op.set_stream(cur)
        opT.set_stream(side)
        ct.ct_forward(op.h, th, None, X, Y, K)
        with torch.cuda.stream(side):
            ct.ct_adjoint(opT.h, th, None, Ys, Xa, K)
        ct.ct_jac(op.h, th, None, X[0], dth, None, dy)
        ct.ct_jacT(op.h, th, None, None, Ys[0], gt, None)
        join = torch.cuda.Event()
        join.record(side)
        cur.wait_event(join)

    op.set_stream(torch.cuda.current_stream())
    ct.ct_forward(op.h, th, None, X, Y, K)
    ct.ct_adjoint(op.h, th, None, Ys, Xa, K)
    ct.ct_jac(op.h, th, None, X[0], dth, None, dy)
    ct.ct_jacT(op.h, th, None, None, Ys[0], gt, None)
    torch.cuda.synchronize()
    ref = [t.clone() for t in (Y, Xa, dy, gt)]
    for t in (Y, Xa, dy, gt):
        t.zero_()
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        overlapped()  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(cap)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        overlapped()
    op.set_stream(torch.cuda.current_stream())
    for t in (Y, Xa, dy, gt):
        t.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(ref, (Y, Xa, dy, gt)):
        assert torch.equal(a, b)
    op.close()
    opT.close()
