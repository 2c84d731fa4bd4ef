"""Seeded synthetic workloads for point-set geodesic shooting.

This module only draws point clouds, momenta and targets; it contains none of
the shooting arithmetic, so both the CUDA path's tests and the CPU oracle can
use it.  Geometries follow the kinds of shapes the paper evaluates on (thin
bent sheets, Sec. 3.1 Fig. 2c; closed cortical-like surfaces, Sec. 3.2):

* ``ellipsoid``  -- points on an ellipsoid surface (semi-axes 20, 15, 10 mm)
  with N(0, 0.5^2) jitter, momenta iid N(0, 0.1^2);
* ``slab``       -- a 40 x 20 x 3 mm sheet bent on an arc of radius R;
* ``blobs``      -- 8 anisotropic Gaussian blobs (axis std 2-6 mm, random
  rotation) inside a 60 mm cube;
* ``sphere``     -- a bumpy closed surface: unit directions scaled to 50 mm
  with a radial perturbation by 32 spherical bumps.

Momenta (except ``ellipsoid``) and target displacements are smooth random
fields: sums of M plane waves with wavelengths of several sigma, so the flow
is smooth on the kernel scale.  Targets are ``X = q0 + u(q0)`` for such a
field u (the objective's cost does not depend on where X lies).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    q0: np.ndarray          # (N, 3) float64
    p0: np.ndarray          # (N, 3) float64
    X: np.ndarray           # (N, 3) float64 targets
    sigma: float
    T: int
    lam: float = 1.0

    @property
    def N(self) -> int:
        return int(self.q0.shape[0])


def _unit(rng, n):
    u = rng.normal(size=(n, 3))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


def smooth_field(x, rng, wavelength, amp, M=8):
    """Sum of M random plane waves, wavelengths in [1, 3] x ``wavelength``,
    random directions, phases and vector coefficients; RMS about ``amp``."""
    dirs = _unit(rng, M)
    lam = wavelength * rng.uniform(1.0, 3.0, size=M)
    k = dirs * (2.0 * math.pi / lam)[:, None]
    phase = rng.uniform(0.0, 2.0 * math.pi, size=M)
    coef = rng.normal(size=(M, 3)) * math.sqrt(2.0 / M)
    s = np.sin(x @ k.T + phase[None, :])          # (N, M)
    return amp * (s @ coef)


def ellipsoid_points(rng, n, axes=(20.0, 15.0, 10.0), jitter=0.5):
    """Uniform by area on the ellipsoid surface (rejection on the area
    element of the map u -> axes * u), plus iid N(0, jitter^2)."""
    a = np.asarray(axes, float)
    out, have = [], 0
    wmax = max(a[0] * a[1], a[0] * a[2], a[1] * a[2])
    while have < n:
        u = _unit(rng, 4 * n)
        w = np.sqrt((u[:, 0] * a[1] * a[2]) ** 2 + (u[:, 1] * a[0] * a[2]) ** 2
                    + (u[:, 2] * a[0] * a[1]) ** 2)
        keep = rng.random(len(u)) < w / wmax
        out.append(u[keep] * a)
        have += int(keep.sum())
    x = np.concatenate(out)[:n]
    return x + rng.normal(scale=jitter, size=x.shape)


def slab_points(rng, n, R=30.0, size=(40.0, 20.0, 3.0)):
    """Uniform in a size[0] x size[1] x size[2] sheet, bent on radius R."""
    L, W, H = size
    x = rng.uniform([0.0, 0.0, -H / 2], [L, W, H / 2], size=(n, 3))
    th = (x[:, 0] - L / 2) / R
    return np.stack([(R + x[:, 2]) * np.sin(th), x[:, 1],
                     (R + x[:, 2]) * np.cos(th) - R], axis=1)


def blob_points(rng, n, nblobs=8, box=60.0):
    """Equal-weight mixture of anisotropic Gaussian blobs (axis std 2-6 mm,
    random rotation, centres in [12, 48]^3), rejected outside [0, box]^3."""
    centres = rng.uniform(12.0, 48.0, size=(nblobs, 3))
    stds = rng.uniform(2.0, 6.0, size=(nblobs, 3))
    rots = []
    for _ in range(nblobs):
        qm, r = np.linalg.qr(rng.normal(size=(3, 3)))
        rots.append(qm * np.sign(np.diag(r))[None, :])
    out, have = [], 0
    while have < n:
        k = rng.integers(0, nblobs, size=2 * n)
        z = rng.normal(size=(2 * n, 3)) * stds[k]
        x = centres[k] + np.einsum("nij,nj->ni", np.stack(rots)[k], z)
        x = x[np.all((x >= 0.0) & (x <= box), axis=1)]
        out.append(x)
        have += len(x)
    return np.concatenate(out)[:n]


def sphere_points(rng, n, radius=50.0, nbumps=32, width=0.3, bump=0.05):
    """Directions uniform on S^2, radius 50 (1 + sum_k a_k b_k(u)) with
    bumps b_k(u) = exp(-|u - c_k|^2 / (2 width^2)), a_k ~ U[-bump, bump]."""
    u = _unit(rng, n)
    c = _unit(rng, nbumps)
    a = rng.uniform(-bump, bump, size=nbumps)
    r = np.ones(n)
    for k in range(nbumps):
        r += a[k] * np.exp(-np.sum((u - c[k]) ** 2, axis=1) / (2.0 * width ** 2))
    return radius * u * r[:, None]


# Momentum amplitudes give displacements of roughly 0.1-1 mm at each
# geometry's typical density (they only set how far the points move).
_SPECS = {
    "ellipsoid": dict(sigma=3.0, T=10, lam=1.0),
    "slab": dict(sigma=2.0, T=20, lam=1.0, p_amp=1.5e-3, u_amp=1.0),
    "blobs": dict(sigma=1.5, T=20, lam=1.0, p_amp=2.0e-4, u_amp=1.0),
    "sphere": dict(sigma=1.0, T=40, lam=1.0, p_amp=5.0e-3, u_amp=1.0),
}

# The five benchmark configurations (name -> geometry, N, seed).
CONFIGS = {
    "ellipsoid1k": ("ellipsoid", 1000, 1001),
    "slab20k": ("slab", 20000, 1002),
    "blobs100k": ("blobs", 100000, 1003),
    "sphere1m": ("sphere", 1000000, 1005),
}


def make(geometry: str, n: int, seed: int, **over) -> Workload:
    """One workload of ``geometry`` with ``n`` points from ``seed``."""
    spec = dict(_SPECS[geometry])
    spec.update(over)
    rng = np.random.default_rng(seed)
    sigma = float(spec["sigma"])
    if geometry == "ellipsoid":
        q0 = ellipsoid_points(rng, n)
        p0 = rng.normal(scale=0.1, size=(n, 3))
        X = q0 + smooth_field(q0, rng, 4.0 * sigma, 0.5)
    else:
        if geometry == "slab":
            q0 = slab_points(rng, n, R=float(spec.get("R", 30.0)))
        elif geometry == "blobs":
            q0 = blob_points(rng, n)
        elif geometry == "sphere":
            q0 = sphere_points(rng, n)
        else:
            raise ValueError(geometry)
        p0 = smooth_field(q0, rng, 4.0 * sigma, float(spec["p_amp"]))
        X = q0 + smooth_field(q0, rng, 6.0 * sigma, float(spec["u_amp"]))
    return Workload(f"{geometry}{n}", q0, p0, X, sigma, int(spec["T"]), float(spec["lam"]))


def config(name: str, n: int | None = None) -> Workload:
    """A named benchmark configuration, optionally at a smaller ``n`` (same
    geometry, seed and parameters)."""
    geom, n0, seed = CONFIGS[name]
    return make(geom, n0 if n is None else n, seed)


def batch(subjects: int = 64, nmin: int = 5000, nmax: int = 40000, seed: int = 1004,
          sigma: float = 2.0, T: int = 20, lam: float = 1.0):
    """Batched registration workload: ``subjects`` slab-shaped clouds with N
    log-uniform in [nmin, nmax] and bending radius U[20, 40] mm.  Returns
    (list of Workload, offsets int64[S+1])."""
    rng = np.random.default_rng(seed)
    ns = np.round(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=subjects))).astype(int)
    radii = rng.uniform(20.0, 40.0, size=subjects)
    ws = []
    for s in range(subjects):
        w = make("slab", int(ns[s]), seed * 1000 + s, R=float(radii[s]), sigma=sigma, T=T, lam=lam)
        ws.append(w)
    offsets = np.zeros(subjects + 1, np.int64)
    offsets[1:] = np.cumsum(ns)
    return ws, offsets
