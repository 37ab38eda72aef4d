"""The allocation-free entry point ct_jacT_noalloc, through the C ABI.

Some callers cannot allocate device memory (a host application that owns all
of it through its own pool, a service whose budget is fixed after start-up);
ct_jacT_noalloc serves them with a static device workspace.  Its results must
equal those of ct_jacT, the entry point it mirrors, on two calls in a row --
the second with another geometry, so a stale workspace from the first call
would show.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_06336_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(N, V, seed):
    rng = np.random.default_rng(seed)
    B = synth.n_bins(N)
    theta = torch.tensor(synth.random_angles(V, rng), dtype=torch.float64, device="cuda")
    delta = torch.tensor(rng.normal(0, 0.5, V), dtype=torch.float64, device="cuda")
    x = torch.tensor(rng.uniform(size=N * N), dtype=torch.float32, device="cuda")
    r = torch.tensor(rng.standard_normal(V * B), dtype=torch.float32, device="cuda")
    return N, B, V, theta, delta, x, r


def _rel(a, b):
    return float((a - b).norm() / b.norm())


def test_noalloc_matches_ct_jacT_on_two_calls_in_a_row():
    from paper_2605_06336_gb300 import ct
    ct.load_library()
    for N, V, seed in ((64, 60, 1), (200, 150, 2)):
        N, B, V, theta, delta, x, r = _case(N, V, seed)
        op = ct.CTOperator(N, B, V, max_batch=1, dtype=torch.float32)
        gt_ref, gd_ref = op.jacT(x, theta, r, delta, want_delta=True)
        gt = torch.full((V,), float("nan"), dtype=torch.float64, device="cuda")
        gd = torch.full((V,), float("nan"), dtype=torch.float64, device="cuda")
        ct.ct_jacT_noalloc(N, B, V, theta, delta, x, r, gt, gd)
        torch.cuda.synchronize()
        assert _rel(gt, gt_ref) <= 1e-5
        assert _rel(gd, gd_ref) <= 1e-5
        op.close()


def test_noalloc_rejects_sizes_beyond_its_workspace():
    from paper_2605_06336_gb300 import ct
    lib = ct.load_library()
    rc = lib.ct_jacT_noalloc(ct.NOALLOC_MAX_N + 1, 8, 4, ctypes.c_void_p(1), None, ctypes.c_void_p(1),
                             ctypes.c_void_p(1), ctypes.c_void_p(1), None, None)
    assert rc == ct.CT_ERR_ARG
    with pytest.raises(ValueError):
        ct.ct_jacT_noalloc(ct.NOALLOC_MAX_N + 1, 8, 4, None, None, None, None, None, None)
