"""The oracle still reproduces its stored regression fixtures (tests/golden/).

The fixtures were written by tests/golden/make_golden.py from the oracle alone;
the paper prints no worked example to store instead.  A failure here means the
oracle's arithmetic changed: the change must name the passage (or the reading
of it) that justifies it, and the fixtures are then rewritten by that script.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import nlrmm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_small.json")


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _close(a, b, rtol):
    a, b = np.asarray(a, float), np.asarray(b, float)
    assert a.shape == b.shape
    assert np.linalg.norm(a - b) <= rtol * max(np.linalg.norm(b), 1e-300), (np.abs(a - b).max(), np.abs(b).max())


@pytest.mark.parametrize("case", ["parallel", "fan"])
def test_operators_reproduce_their_fixture(golden, case):
    c = golden[case]
    geo = c["geometry"]
    g = oracle.Geometry(geo["N"], geo["B"], geo["V"], fan_D=geo["fan_D"])
    th, dl = np.array(c["theta"]), np.array(c["delta"])
    x, y = np.array(c["x"]), np.array(c["y"])
    _close(oracle.forward(g, th, x, dl), c["forward"], 1e-13)
    _close(oracle.adjoint(g, th, y, dl), c["adjoint"], 1e-13)
    _close(oracle.jac(g, th, x, np.array(c["dtheta"]), dl, np.array(c["ddelta"])), c["jac"], 1e-13)
    gt, gd = oracle.jacT(g, th, x, y, dl)
    _close(gt, c["jacT_theta"], 1e-13)
    _close(gd, c["jacT_delta"], 1e-13)


def test_solver_reproduces_its_fixture(golden):
    c = golden["solver"]
    geo, op = c["geometry"], c["options"]
    g = oracle.Geometry(geo["N"], geo["B"], geo["V"])
    opts = nlrmm.Options(k_min=op["k_min"], k_max=op["k_max"], noise_norm=c["noise_norm"],
                         outer_iters=op["outer_iters"], stop_on_convergence=False)
    u, th, hist = nlrmm.NLRMMGKS(g, np.array(c["b"]), opts).solve(
        np.array(c["theta0"]), u_true=np.array(c["u_true"]), theta_true=np.array(c["theta_true"]))
    _close(hist.lam, c["lambda"], 1e-9)   # the bisection's last halvings sit at ~1e-17 in log10(lambda)
    _close(hist.rre, c["rre"], 1e-9)
    _close(th, c["theta"], 1e-12)
    _close(u, c["u"], 1e-9)
