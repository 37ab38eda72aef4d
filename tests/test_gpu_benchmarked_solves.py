"""The FP32 NL-RMM-GKS solves the benchmark times, against the FP64 oracle's.

The 256^2 / 180-view workload (30 outer iterations) and the 16-frame dynamic
workload with ANISO-TV (10 outer iterations, recycling space of 50 vectors):
the oracle's solves of the same data take minutes to an hour on the host, so
tests/golden/make_solver_golden.py stores their results (oracle only, the
Armijo searches with the noise floor of an FP32 misfit).  Here the data are
rebuilt with the oracle forward, checked against the stored norm, and solved
by the FP32 GPU form (FP32 operators, FP64 small algebra, batched basis
projection, CUDA graphs): the final relative reconstruction error must match
the oracle's within 1e-3 (relative), and the angle error may not exceed the
oracle's by more than 5 %.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "oracle_solves.json")


def _stored():
    if not os.path.exists(GOLDEN):
        return {}
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["C2", "C4"])
def test_fp32_benchmarked_solve_reaches_the_oracle(name):
    ref = _stored().get(name)
    if ref is None:
        pytest.skip(f"no stored oracle solve for {name}")
    import sys
    sys.path.insert(0, os.path.join(HERE, "golden"))
    from make_solver_golden import data
    from paper_2605_06336_gb300 import ct
    w, g, u, b, nn = data(name)
    assert abs(np.linalg.norm(b) - ref["b_norm"]) <= 1e-12 * ref["b_norm"]
    dev = lambda a, t: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    op = ct.CTOperator(w.N, w.B, w.V, w.views_per_frame, max_batch=8, dtype=torch.float32)
    opts = {k: (int(v) if isinstance(v, bool) else v) for k, v in ref["options"].items()}
    x, th, st = op.solve(dev(b, torch.float32), dev(w.theta_nominal, torch.float64),
                         x_true=dev(u, torch.float32), noise_norm=nn, stop_on_convergence=0, **opts)
    rre_gpu, rre_orc = st["rre"][-1], ref["rre"][-1]
    assert abs(rre_gpu - rre_orc) <= 1e-3 * rre_orc, (rre_gpu, rre_orc)
    ang = float(np.linalg.norm(th.cpu().numpy() - w.theta_true) / np.linalg.norm(w.theta_true))
    assert ang <= 1.05 * ref["angle_err"][-1], (ang, ref["angle_err"][-1])
