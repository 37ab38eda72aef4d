"""GPU streaming NL-RMM-GKS (nlrmm_stream_solve) against the FP64 oracle's stream_solve.

Views are drawn into blocks without replacement (Sec. 2.4); each block gets its
own handle.
* FP64 operators, Enlarge early stop off: the per-pass lambda of the last
  block, the per-pass RRE, the final image and every block's angles follow the
  oracle's iterates;
* FP32 operators + FP64 small algebra, with the paper's tol_1 early stop of
  Alg. "Enlarge" on: the final RRE matches the oracle's within 1e-3 (relative)
  and the angle error is no worse than 1.05x; both sides apply the Armijo
  noise floor of an FP32 misfit (unit roundoff 2^-24);
* inconsistent blocks (another image size) are refused.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import nlrmm
from paper_2605_06336_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def streaming_problem(N, V, nblocks, seed, noise=0.01, sigma_deg=0.5):
    rng = np.random.default_rng(seed)
    B = synth.n_bins(N)
    g = oracle.Geometry(N, B, V)
    th_nom = np.sort(synth.random_angles(V, rng))
    th_true = th_nom + rng.normal(0, math.radians(sigma_deg), V)
    u_true = synth.rasterize(N, synth.random_ellipses(N, 4, rng)).ravel()
    b_true = oracle.forward(g, th_true, u_true).reshape(V, B)
    e = rng.standard_normal(b_true.shape)
    e *= noise * np.linalg.norm(b_true) / np.linalg.norm(e)
    blocks = []
    for ix in np.array_split(rng.permutation(V), nblocks):
        ix = np.sort(ix)
        blocks.append(dict(g=oracle.Geometry(N, B, len(ix)), b=(b_true[ix] + e[ix]).ravel(),
                           th0=th_nom[ix], tht=th_true[ix], nn=float(np.linalg.norm(e[ix]))))
    return blocks, u_true


def _run_both(blocks, u_true, dtype, passes, **kw):
    from paper_2605_06336_gb300 import ct
    orc = [nlrmm.NLRMMGKS(bk["g"], bk["b"], nlrmm.Options(noise_norm=bk["nn"], stop_on_convergence=False,
                                                           **{k: v for k, v in kw.items()}))
           for bk in blocks]
    u_o, th_o, h_o = nlrmm.stream_solve(orc, [bk["th0"] for bk in blocks], passes=passes, u_true=u_true,
                                        theta_true=[bk["tht"] for bk in blocks])
    ops = [ct.CTOperator(bk["g"].N, bk["g"].B, bk["g"].V, max_batch=8, dtype=dtype) for bk in blocks]
    x, th, st = ct.stream_solve(ops, [dev(bk["b"], dtype) for bk in blocks], [dev(bk["th0"]) for bk in blocks],
                                [bk["nn"] for bk in blocks], x_true=dev(u_true, dtype), outer_iters=passes,
                                stop_on_convergence=0, **{k: (int(v) if isinstance(v, bool) else v)
                                                          for k, v in kw.items()})
    return (u_o, th_o, h_o), (x, th, st)


def test_fp64_streaming_follows_the_oracle_iterates():
    blocks, u_true = streaming_problem(32, 36, 3, seed=31)
    (u_o, th_o, h_o), (x, th, st) = _run_both(blocks, u_true, torch.float64, passes=3, k_min=5, k_max=15, tol1=0.0)
    assert st["passes"] == 3
    assert st["enlarge_steps"] == h_o.enlarge_steps
    # 9 block visits, each ending in Gauss-Newton steps whose quotient -g/|J|^2
    # amplifies the rounding differences of the two FP64 paths: 1e-6 relative
    # on lambda, RRE and the image, 1e-7 rad on the angles
    np.testing.assert_allclose(st["lambda"], h_o.lam, rtol=1e-6)
    np.testing.assert_allclose(st["rre"], h_o.rre, rtol=1e-6)
    xu = x.cpu().numpy()
    assert np.linalg.norm(xu - u_o) <= 1e-6 * np.linalg.norm(u_o)
    for a, b in zip(th, th_o):
        assert np.max(np.abs(a.cpu().numpy() - b)) <= 1e-7


def test_fp32_streaming_reaches_the_oracle_reconstruction_error():
    # 4 passes x 4 blocks with the paper's tol_1 early stop on (default 1e-3);
    # the oracle runs the Armijo searches with the noise floor of an FP32
    # misfit, as the FP32 GPU form does, so that neither side takes steps whose
    # acceptance is decided by rounding.
    blocks, u_true = streaming_problem(64, 90, 4, seed=32)
    (u_o, th_o, h_o), (x, th, st) = _run_both(blocks, u_true, torch.float32, passes=4, armijo_eps=2.0 ** -24)
    rre_gpu, rre_orc = st["rre"][-1], h_o.rre[-1]
    assert abs(rre_gpu - rre_orc) <= 1e-3 * rre_orc, (rre_gpu, rre_orc)
    err = np.concatenate([t.cpu().numpy() - bk["tht"] for t, bk in zip(th, blocks)])
    ang_gpu = np.linalg.norm(err) / np.linalg.norm(np.concatenate([bk["tht"] for bk in blocks]))
    assert ang_gpu <= 1.05 * h_o.angle_err[-1], (ang_gpu, h_o.angle_err[-1])


def test_streaming_refuses_inconsistent_blocks():
    from paper_2605_06336_gb300 import ct
    a = ct.CTOperator(16, 23, 6, max_batch=2, dtype=torch.float32)
    b = ct.CTOperator(18, 26, 6, max_batch=2, dtype=torch.float32)
    with pytest.raises(ct.CTError) as e:
        ct.nlrmm_stream_solve([a.h, b.h], [torch.zeros(6 * 23, device="cuda"), torch.zeros(6 * 26, device="cuda")],
                              [torch.zeros(6, dtype=torch.float64, device="cuda")] * 2, None, [1.0, 1.0],
                              torch.zeros(256, device="cuda"))
    assert e.value.code == ct.CT_ERR_ARG
