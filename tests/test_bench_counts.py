"""The algorithmic work count behind the bench's roofline.

bench.interp_steps_per_image counts the (ray, sample) pairs with -1 < q < N,
the interpolation steps whose two taps the roofline charges as 8 gathered bytes.
Here the same count comes from the oracle's dense matrix instead: a sample of a
row-marched ray lies inside the image exactly when that ray has a nonzero
entry in the sample's image row (columns for column-marched rays).
"""
import math
import types

import numpy as np

import bench
import oracle
from paper_2605_06336_gb300 import synth


def test_interpolation_step_count_matches_the_dense_matrix():
    rng = np.random.default_rng(12)
    N, V = 12, 16
    B = synth.n_bins(N)
    theta = synth.random_angles(V, rng, avoid_diagonal=1e-3)
    w = types.SimpleNamespace(N=N, B=B, theta_true=theta)
    A = oracle.dense_matrix(oracle.Geometry(N, B, V), theta).reshape(V, B, N, N)
    count = 0
    for v in range(V):
        rows = abs(math.cos(theta[v])) >= abs(math.sin(theta[v]))
        nz = A[v] != 0.0                                   # [B][N][N]
        count += int((nz.any(axis=2) if rows else nz.any(axis=1)).sum())
    assert bench.interp_steps_per_image(w) == count
