"""The C part of the oracle runs clean under AddressSanitizer and UBSan.

A sanitized copy of oracle/ct_oracle.c is built into a temporary folder and
driven, in a child process with the ASan runtime preloaded, through the
oracle's own Python wrappers on edge cases: one-pixel and one-bin
geometries, an empty frame, views on the Joseph switch angles and outside
[0, pi), offsets that push every ray off the image, and fan beams with the
source close in and far away.  Skipped where gcc has no sanitizer runtime.
"""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import math, sys
    import numpy as np
    import oracle
    oracle._LIB = sys.argv[1]          # the sanitized build (newer than the source: no rebuild)
    from paper_2605_06336_gb300 import synth
    rng = np.random.default_rng(0)
    calls = 0
    for N in (1, 2, 3, 8, 17):
        for B in (1, 2, synth.n_bins(N), 2 * N + 7):
            for fan in (None, 0.75 * max(N, B) + 3.0, 1e6):
                V = 7
                g = oracle.Geometry(N, B, V, views_per_frame=[3, 0, 4] if N > 2 else None, fan_D=fan)
                th = np.array([0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4, -1.0, 7.0, 2.9])
                dl = np.array([0.0, 0.5, -0.5, 100.0, -100.0, 1e-9, 3.3])
                x = rng.standard_normal(g.n)
                y = rng.standard_normal(g.m)
                for d in (None, dl):
                    oracle.forward(g, th, x, d)
                    oracle.adjoint(g, th, y, d)
                    oracle.dsample(g, th, x, d)
                    oracle.jac(g, th, x, rng.standard_normal(V), d, None if d is None else rng.standard_normal(V))
                    oracle.jacT(g, th, x, y, d)
                    calls += 5
    print("calls", calls)
""")


def _runtime():
    try:
        p = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True, check=True)
    except (OSError, subprocess.CalledProcessError):
        return None
    path = p.stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_oracle_is_clean_under_sanitizers(tmp_path):
    asan = _runtime()
    if asan is None:
        pytest.skip("gcc has no AddressSanitizer runtime here")
    lib = tmp_path / "liboracle_ct_sanitized.so"
    src = os.path.join(ROOT, "oracle", "ct_oracle.c")
    subprocess.run(["gcc", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
                    "-std=c99", "-fPIC", "-shared", "-o", str(lib), src, "-lm"], check=True)
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD, str(lib)], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    assert "calls 600" in r.stdout, r.stdout
