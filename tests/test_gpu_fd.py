"""Finite differences of the CUDA path's own objective against its adjoint
gradient (Eq. 2 differentiated by the backward stage, Sec. 2.1-2.2), on the
20k slab at its stated T = 20, exact mode, along 16 random unit momentum
directions (the slab configuration's check).

Step choice.  H is quadratic in p0, so the central difference's truncation
error, eps^2 / 6 times the third derivative of E along v, comes from the
data term alone; with the FP64 oracle on a 3000-point slab (same sigma, T
and amplitudes) it was about 1e-6 of grad.v at eps = 0.1 |p0| (|p0| the
Euclidean norm of all 3N momenta), shrinking by 4 per halving.  The CUDA
path's E is formed from FP32-pair sums; its rounding moves E by a few 1e-8
relative, mostly as a bias that changes smoothly with p0 and cancels in the
difference, so the noise left is far below the pessimistic bound
2 * 3e-8 * |E| / eps printed beside the errors.  eps = 0.1 |p0| and eps / 2
are taken.
"""
import numpy as np
import pytest

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt, npy

pytestmark = pytest.mark.gpu


def test_fd_gradient_slab20k():
    w = inputs.config("slab20k")
    q0, X = dt(w.q0), dt(w.X)
    E0, g, _ = gs.shoot_grad(q0, dt(w.p0), X, w.sigma, w.T, w.lam)
    g = npy(g)
    E0 = float(npy(E0)[0])
    rng = np.random.default_rng(1002 + 2)
    eps = 0.1 * float(np.linalg.norm(w.p0))

    def E_at(p):
        return float(npy(gs.shoot_grad(q0, dt(p), X, w.sigma, w.T, w.lam)[0])[0])

    rows = []
    for _ in range(16):
        v = rng.normal(size=w.p0.shape)
        v /= np.linalg.norm(v)
        d = float(np.sum(g * v))
        fd = [(E_at(w.p0 + e * v) - E_at(w.p0 - e * v)) / (2 * e) for e in (eps, eps / 2)]
        rows.append((d, fd[0], fd[1]))
    rows = np.array(rows)
    scale = np.abs(rows[:, 0]).max()
    err1 = np.abs(rows[:, 1] - rows[:, 0]) / scale
    err2 = np.abs(rows[:, 2] - rows[:, 0]) / scale
    noise = 2 * 3e-8 * abs(E0) / (eps / 2) / scale
    print(f"\nslab20k exact, T={w.T}: |E| {abs(E0):.4e}, eps {eps:.3e}; FD vs grad.v, relative to "
          f"max|grad.v| {scale:.4e}: step eps max {err1.max():.2e}, step eps/2 max "
          f"{err2.max():.2e} (tol 1e-4); noise bound at eps/2 {noise:.1e}")
    assert err2.max() <= 1e-4
