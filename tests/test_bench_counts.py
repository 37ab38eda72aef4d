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


def test_launches_per_step_follow_the_launch_shapes():
    """Kernels per bench step: the forward block's, the sinograms' and J's layouts,
    J^T's view-table step, the forward kernel(s), the transpose kernel(s), JVP, VJP
    and the per-view sums; one forward launch per group width the batch of 8 needs,
    and a combining kernel for a staged forward split over CTAs."""
    base = [4, 4, 1, 8, 4, 4, 1, 0, 0, 8, 2, 1]
    assert bench.launches_per_step(base) == 9
    assert bench.launches_per_step(base[:11] + [0]) == 9      # pair images: the same launches
    assert bench.launches_per_step([8, 2, 1] + base[3:]) == 9
    assert bench.launches_per_step([1, 2, 1] + base[3:]) == 9  # 8 groups of 1, one launch
    staged = [4, 2, 4, 8, 4, 4, 1, 4, 0, 8, 2, 0]
    assert bench.launches_per_step(staged) == 10             # + the segment combine
    assert bench.launches_per_step([4, 1, 4, 8, 4, 4, 1, 4, 0, 8, 2, 0]) == 9  # staged, one CTA per ray
