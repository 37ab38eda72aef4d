"""Writes the oracle regression fixtures of this folder.

Every value here comes from the FP64 oracle (``oracle/``) on seeded synthetic
inputs (``paper_2605_06336_gb300/synth.py``); nothing is read from the CUDA
path.  The paper prints no worked example of the operator or the solver (its
tables are experiments on data that is not available), so these fixtures are
regression guards of the oracle itself, whose correctness is established by
the pins in ``tests/test_oracle_*.py``: a later change to the oracle's
arithmetic shows up here and must name its justification.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import nlrmm  # noqa: E402
from paper_2605_06336_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def operator_case(fan_D=None):
    """8 x 8 image, 6 views with offsets: H x, H^T y, J_theta dtheta + J_delta ddelta, J^T y."""
    rng = np.random.default_rng(20260605)
    N, V = 8, 6
    B = synth.n_bins(N)
    g = oracle.Geometry(N, B, V, fan_D=fan_D)
    theta = synth.random_angles(V, rng, avoid_diagonal=1e-2)
    delta = rng.normal(0.0, 0.5, V)
    x = synth.rasterize(N, synth.random_ellipses(N, 3, rng)).ravel()
    y = rng.standard_normal(g.m)
    dth, ddl = rng.standard_normal(V), rng.standard_normal(V)
    gt, gd = oracle.jacT(g, theta, x, y, delta)
    return {
        "geometry": {"N": N, "B": B, "V": V, "fan_D": fan_D},
        "theta": theta.tolist(), "delta": delta.tolist(), "x": x.tolist(), "y": y.tolist(),
        "dtheta": dth.tolist(), "ddelta": ddl.tolist(),
        "forward": oracle.forward(g, theta, x, delta).tolist(),
        "adjoint": oracle.adjoint(g, theta, y, delta).tolist(),
        "jac": oracle.jac(g, theta, x, dth, delta, ddl).tolist(),
        "jacT_theta": gt.tolist(), "jacT_delta": gd.tolist(),
    }


def solver_case():
    """12 x 12 image, 10 views, 5 % noise: 3 outer iterations of NL-RMM-GKS with the discrepancy principle."""
    rng = np.random.default_rng(20260606)
    N, V = 12, 10
    g = oracle.Geometry(N, synth.n_bins(N), V)
    th_nom = np.sort(rng.uniform(0.0, math.pi, V))
    th_true = th_nom + rng.normal(0.0, math.radians(0.5), V)
    u_true = synth.rasterize(N, synth.random_ellipses(N, 3, rng)).ravel()
    b_true = oracle.forward(g, th_true, u_true)
    e = rng.standard_normal(g.m)
    e *= 0.05 * np.linalg.norm(b_true) / np.linalg.norm(e)
    b = b_true + e
    opts = nlrmm.Options(k_min=4, k_max=20, noise_norm=float(np.linalg.norm(e)), outer_iters=3,
                         stop_on_convergence=False)
    u, th, hist = nlrmm.NLRMMGKS(g, b, opts).solve(th_nom, u_true=u_true, theta_true=th_true)
    return {
        "geometry": {"N": N, "B": g.B, "V": V},
        "options": {"k_min": 4, "k_max": 20, "outer_iters": 3, "noise": 0.05},
        "b": b.tolist(), "theta0": th_nom.tolist(), "noise_norm": float(np.linalg.norm(e)),
        "u_true": u_true.tolist(), "theta_true": th_true.tolist(),
        "lambda": [float(v) for v in hist.lam], "rre": hist.rre, "theta": th.tolist(), "u": u.tolist(),
    }


def main():
    cases = {"parallel": operator_case(), "fan": operator_case(fan_D=20.0), "solver": solver_case()}
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(cases, f, indent=0)
        f.write("\n")


if __name__ == "__main__":
    main()
