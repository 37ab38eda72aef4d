"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds input generation only (phantoms, angle sets, noise
directions, workload shapes).  It contains none of the operator or solver
arithmetic, so it can feed both the CUDA path and the CPU oracle.

Recipe (random ellipses stand in for the paper's Shepp-Logan / Moving-MNIST
data, which are not available):
  * ellipse centres uniform in the disc of radius 0.35 N, semi-axes
    U[0.05 N, 0.25 N], rotation U[0, pi), intensity U[0, 1]; overlaps add;
    rasterised at pixel centres with 4x4 supersampling;
  * pixel (i, j) centre at x = j - (N-1)/2, y = (N-1)/2 - i;
  * B = ceil(sqrt(2) N) detector bins of unit width.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20260605


def n_bins(N: int) -> int:
    return int(math.ceil(math.sqrt(2.0) * N))


@dataclass
class Ellipse:
    cx: float
    cy: float
    a: float      # semi-axis along direction phi
    b: float      # semi-axis perpendicular to phi
    phi: float
    rho: float    # intensity


def random_ellipses(N: int, count: int, rng: np.random.Generator) -> list[Ellipse]:
    out = []
    for _ in range(count):
        r = 0.35 * N * math.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2.0 * math.pi)
        a = rng.uniform(0.05 * N, 0.25 * N)
        b = rng.uniform(0.05 * N, 0.25 * N)
        phi = rng.uniform(0.0, math.pi)
        rho = rng.uniform(0.0, 1.0)
        out.append(Ellipse(r * math.cos(ang), r * math.sin(ang), a, b, phi, rho))
    return out


def rasterize(N: int, ellipses: list[Ellipse], supersample: int = 4, shift=(0.0, 0.0)) -> np.ndarray:
    """N x N image (float64, row-major) of the ellipses, averaged over s x s sub-samples per pixel."""
    img = np.zeros((N, N))
    h = 0.5 * (N - 1)
    offs = (np.arange(supersample) + 0.5) / supersample - 0.5
    for e in ellipses:
        cx, cy = e.cx + shift[0], e.cy + shift[1]
        rad = max(e.a, e.b) + 1.0
        j_lo = max(0, int(math.floor(cx - rad + h)))
        j_hi = min(N - 1, int(math.ceil(cx + rad + h)))
        i_lo = max(0, int(math.floor(h - (cy + rad))))
        i_hi = min(N - 1, int(math.ceil(h - (cy - rad))))
        if j_lo > j_hi or i_lo > i_hi:
            continue
        jj = np.arange(j_lo, j_hi + 1)
        ii = np.arange(i_lo, i_hi + 1)
        cphi, sphi = math.cos(e.phi), math.sin(e.phi)
        acc = np.zeros((ii.size, jj.size))
        for dy in offs:
            y = (h - ii)[:, None] - dy - cy
            for dx in offs:
                x = (jj - h)[None, :] + dx - cx
                u = (x * cphi + y * sphi) / e.a
                w = (-x * sphi + y * cphi) / e.b
                acc += (u * u + w * w) <= 1.0
        img[i_lo:i_hi + 1, j_lo:j_hi + 1] += e.rho * acc / (supersample * supersample)
    return img


def unit_noise(m: int, rng: np.random.Generator) -> np.ndarray:
    """Standard normal direction; the caller scales it to the stated noise level."""
    return rng.standard_normal(m)


@dataclass
class Workload:
    name: str
    N: int
    B: int
    views_per_frame: list[int]
    theta_nominal: np.ndarray        # (V,) radians, what the solver starts from
    theta_true: np.ndarray           # (V,) radians, used to simulate the data
    delta_true: np.ndarray | None    # (V,) detector offsets in pixels, or None
    images: np.ndarray               # (F, N, N) true images
    noise_level: float
    noise_dir: np.ndarray            # (V*B,) unit-normal direction
    batch: int = 1                   # Krylov block width used for the batched operator
    outer_iters: int = 20
    extra: dict = field(default_factory=dict)

    @property
    def F(self):
        return len(self.views_per_frame)

    @property
    def V(self):
        return int(sum(self.views_per_frame))


def _perturb(rng, nominal, sigma_deg):
    return nominal + rng.normal(0.0, math.radians(sigma_deg), size=nominal.shape)


def make_workload(name: str, scale: float = 1.0) -> Workload:
    """The five synthetic workloads.

    ``scale`` < 1 shrinks the image side (and bins, views) for quick tests of
    the same recipe; the benchmark and the full-size checks use scale = 1.
    """
    idx = {"C1": 1, "C2": 2, "C3": 3, "C4": 4, "C5": 5}[name]
    rng = np.random.default_rng(SEED_BASE + idx)

    def S(n):
        return max(8, int(round(n * scale)))

    if name == "C1":
        N, V = S(64), S(90)
        B = n_bins(N)
        nominal = np.sort(rng.uniform(0.0, math.pi, V))
        true = _perturb(rng, nominal, 0.5)
        imgs = rasterize(N, random_ellipses(N, 5, rng))[None]
        return Workload(name, N, B, [V], nominal, true, None, imgs, 0.01, unit_noise(V * B, rng),
                        batch=8, outer_iters=20)
    if name == "C2":
        N, V = S(256), S(180)
        B = n_bins(N)
        nominal = np.sort(rng.uniform(0.0, math.pi, V))
        true = _perturb(rng, nominal, 1.0)
        imgs = rasterize(N, random_ellipses(N, 10, rng))[None]
        return Workload(name, N, B, [V], nominal, true, None, imgs, 0.01, unit_noise(V * B, rng),
                        batch=8, outer_iters=30)
    if name == "C3":
        N, V = S(512), S(360)
        B = n_bins(N)
        nominal = np.arange(V) * (math.pi / V)
        true = _perturb(rng, nominal, 1.0)
        delta = rng.normal(0.0, 0.5, size=V)
        imgs = rasterize(N, random_ellipses(N, 10, rng))[None]
        return Workload(name, N, B, [V], nominal, true, delta, imgs, 0.01, unit_noise(V * B, rng),
                        batch=8, outer_iters=10)
    if name == "C4":
        N, F = S(256), 16
        B = n_bins(N)
        lo, hi = max(2, S(30)), max(3, S(120))
        vpf = [int(v) for v in rng.integers(lo, hi + 1, size=F)]
        V = sum(vpf)
        golden = math.pi * (math.sqrt(5.0) - 1.0) / 2.0
        nominal = np.mod(np.arange(V) * golden, math.pi)
        true = _perturb(rng, nominal, 0.5)
        ells = random_ellipses(N, 10, rng)
        ang = rng.uniform(0.0, 2.0 * math.pi)
        d = (math.cos(ang), math.sin(ang))
        imgs = np.stack([rasterize(N, ells, shift=(t * d[0], t * d[1])) for t in range(F)])
        return Workload(name, N, B, vpf, nominal, true, None, imgs, 0.01, unit_noise(V * B, rng),
                        batch=8, outer_iters=10)
    if name == "C5":
        N, V = S(2048), S(1440)
        B = n_bins(N)
        nominal = np.arange(V) * (math.pi / V)
        true = _perturb(rng, nominal, 0.5)  # sigma^2 = 0.25 deg^2
        imgs = rasterize(N, random_ellipses(N, 40, rng))[None]
        chunks = rng.permutation(V).reshape(12, -1) if V % 12 == 0 else np.array_split(rng.permutation(V), 12)
        w = Workload(name, N, B, [V], nominal, true, None, imgs, 0.005, unit_noise(V * B, rng),
                     batch=8, outer_iters=12)
        w.extra["chunks"] = [np.sort(c) for c in chunks]
        return w
    raise KeyError(name)


def random_angles(V: int, rng: np.random.Generator, avoid_diagonal: float = 1e-6) -> np.ndarray:
    """Random view angles in [0, pi) kept away from odd multiples of pi/4.

    At |cos| = |sin| the Joseph rule switches its marching axis; the two
    sides of a parity check must not be asked to break that tie differently
    in their last bit, so test angles stay ``avoid_diagonal`` away from it.
    """
    th = rng.uniform(0.0, math.pi, V)
    d = np.mod(th - math.pi / 4, math.pi / 2)
    near = np.minimum(d, math.pi / 2 - d) < avoid_diagonal
    th[near] += 10 * avoid_diagonal
    return th
