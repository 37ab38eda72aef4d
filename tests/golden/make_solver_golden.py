"""Writes the oracle's results for the benchmarked NL-RMM-GKS solves.

The FP32 GPU solves that the benchmark times (the 256^2 / 180-view workload,
30 outer iterations; the 16-frame dynamic workload with ANISO-TV, 10 outer
iterations and a recycling space of 50 vectors) are checked against the FP64
oracle's solves of the same data.  Those take minutes (the second about an
hour) on the host, so their results are stored here.  Every value comes from
``oracle/`` on inputs from ``paper_2605_06336_gb300/synth.py``; nothing is
read from the CUDA path.  The oracle runs the Armijo searches with the noise
floor of an FP32 misfit (unit roundoff 2^-24), as the FP32 GPU form does.

Run from the repository root:  python tests/golden/make_solver_golden.py [C2|C4]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import nlrmm  # noqa: E402
from paper_2605_06336_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
PATH = os.path.join(HERE, "oracle_solves.json")
CASES = {
    "C2": dict(outer_iters=30),
    "C4": dict(outer_iters=10, temporal=True, k_max=50),
}


def data(name):
    """Workload, noisy data b = H(theta_true) u_true + e (oracle forward), noise norm."""
    w = synth.make_workload(name)
    g = oracle.Geometry(w.N, w.B, w.V, w.views_per_frame)
    u = w.images.reshape(-1)
    bt = oracle.forward(g, w.theta_true, u)
    e = w.noise_dir * (w.noise_level * np.linalg.norm(bt) / np.linalg.norm(w.noise_dir))
    return w, g, u, bt + e, float(np.linalg.norm(e))


def solve(name):
    w, g, u, b, nn = data(name)
    kw = CASES[name]
    o = nlrmm.Options(noise_norm=nn, stop_on_convergence=False, armijo_eps=2.0 ** -24, **kw)
    t0 = time.time()
    _, th, h = nlrmm.NLRMMGKS(g, b, o).solve(w.theta_nominal, u_true=u, theta_true=w.theta_true)
    return {"options": kw, "armijo_eps": 2.0 ** -24, "b_norm": float(np.linalg.norm(b)), "noise_norm": nn,
            "rre": h.rre, "angle_err": h.angle_err, "lambda": [float(v) for v in h.lam],
            "enlarge_steps": h.enlarge_steps, "theta": th.tolist(), "host_seconds": time.time() - t0}


def main():
    out = json.load(open(PATH)) if os.path.exists(PATH) else {}
    for name in (sys.argv[1:] or list(CASES)):
        out[name] = solve(name)
        with open(PATH, "w") as f:
            json.dump(out, f, indent=0)
            f.write("\n")


if __name__ == "__main__":
    main()
