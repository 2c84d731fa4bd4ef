"""Parity of the exact all-pairs CUDA path (Sec. 2.1: Eq. 1 flow, Euler
shooting, discrete adjoint) with the FP64 oracle, through the C ABI.

Tolerances: positions max |dq(1)| <= 1e-5 sigma; gradients relative L2 <=
1e-4; a single right-hand side within 1e-5 of its own scale (an error of that
size integrated over t in [0, 1] moves points by far less than 1e-5 sigma)."""
import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from paper_1907_04834_gb300._lib import GS_ERR_INVALID_ARG
from gpu_util import dt, npy, max_rel, rel_l2, phi_floor

pytestmark = pytest.mark.gpu

CASES = [("ellipsoid", 1000, 1001), ("slab", 1, 5), ("slab", 2, 6), ("slab", 513, 7),
         ("blobs", 2049, 8), ("slab", 3000, 9)]


@pytest.mark.parametrize("geom,n,seed", CASES)
def test_rhs_matches_oracle(oracle, geom, n, seed):
    w = inputs.make(geom, n, seed)
    F, Phi, cnt = gs.rhs(dt(w.q0), dt(w.p0), w.sigma)
    Fo, Phio, _ = oracle.rhs(w.q0, w.p0, w.sigma)
    assert cnt == (n * n, 0)
    assert max_rel(npy(F), Fo) <= 1e-5
    if n > 1:
        assert max_rel(npy(Phi), Phio, phi_floor(w.p0, w.sigma)) <= 1e-5
    else:
        assert np.all(npy(Phi) == 0)


@pytest.mark.parametrize("geom,n,seed", CASES)
def test_adjoint_rhs_matches_oracle(oracle, geom, n, seed):
    w = inputs.make(geom, n, seed)
    rng = np.random.default_rng(seed)
    al = rng.normal(size=w.q0.shape)
    be = rng.normal(scale=0.1, size=w.q0.shape)
    dA, dB, _ = gs.adj_rhs(dt(w.q0), dt(w.p0), dt(al), dt(be), w.sigma)
    dAo, dBo, _ = oracle.adj_rhs(w.q0, w.p0, al, be, w.sigma)
    assert max_rel(npy(dA), dAo, 1e-12 * np.abs(al).max() * np.abs(w.p0).max() / w.sigma) <= 1e-5
    assert max_rel(npy(dB), dBo) <= 1e-5


@pytest.mark.parametrize("geom,n,seed,T", [("ellipsoid", 1000, 1001, 10), ("slab", 4000, 3, 20),
                                           ("blobs", 3000, 4, 20), ("slab", 1, 5, 7),
                                           ("slab", 2, 6, 3)])
def test_shoot_matches_oracle(oracle, geom, n, seed, T):
    w = inputs.make(geom, n, seed, T=T)
    q1, p1, H = gs.shoot(dt(w.q0), dt(w.p0), w.sigma, w.T, with_H=True)
    q1o, p1o, Ho = oracle.shoot(w.q0, w.p0, w.sigma, w.T)
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma
    assert max_rel(npy(p1), p1o) <= 1e-5
    np.testing.assert_allclose(npy(H), Ho, rtol=1e-6)


def test_full_config1_ellipsoid(oracle):
    """N = 1000 ellipsoid, sigma = 3, T = 10, momenta iid N(0, 0.1^2): q(1),
    p(1) and the Hamiltonian drift against the FP64 oracle."""
    w = inputs.config("ellipsoid1k")
    q1, p1, H = gs.shoot(dt(w.q0), dt(w.p0), w.sigma, w.T, with_H=True)
    q1o, p1o, Ho = oracle.shoot(w.q0, w.p0, w.sigma, w.T)
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma
    Hg = npy(H)
    assert abs((Hg[1] - Hg[0]) - (Ho[1] - Ho[0])) <= 1e-6 * abs(Ho[0])


@pytest.mark.parametrize("geom,n,seed,T", [("slab", 2000, 11, 8), ("blobs", 1500, 12, 6),
                                           ("slab", 3, 13, 4)])
def test_gradient_matches_oracle(oracle, geom, n, seed, T):
    w = inputs.make(geom, n, seed, T=T)
    E, g, q1 = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam)
    Eo, go, q1o = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, w.lam)
    assert rel_l2(npy(g), go) <= 1e-4
    np.testing.assert_allclose(npy(E), Eo, rtol=1e-6)
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma


def test_checkpointing_is_bit_exact():
    """Recomputing the trajectory from checkpoints reproduces every step bit
    for bit, so the gradient equals the store-everything gradient."""
    w = inputs.make("slab", 1800, 21, T=11)
    E0, g0, q0 = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam)
    for ck in (1, 3, 4, 10):
        E1, g1, q1 = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam,
                                   ckpt_every=ck)
        assert torch.equal(g0, g1) and torch.equal(E0, E1) and torch.equal(q0, q1), ck


def test_host_buffers_match_device_buffers():
    w = inputs.make("blobs", 777, 22, T=5)
    Ed, gd, qd = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam)
    c = lambda a: torch.as_tensor(a, dtype=torch.float64)
    Eh, gh, qh = gs.shoot_grad(c(w.q0), c(w.p0), c(w.X), w.sigma, w.T, w.lam)
    assert not gh.is_cuda
    assert torch.equal(gh, gd.cpu()) and torch.equal(Eh, Ed.cpu()) and torch.equal(qh, qd.cpu())


def test_autograd_function():
    w = inputs.make("slab", 500, 23, T=4)
    p0 = dt(w.p0).requires_grad_(True)
    E = gs.energy(p0, dt(w.q0), dt(w.X), w.sigma, w.T, w.lam)
    (2.0 * E).backward()
    _, g, _ = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam)
    assert torch.allclose(p0.grad, 2.0 * g, rtol=0, atol=0)


def test_translation_far_from_origin(oracle):
    """Recentring keeps FP32 positions accurate for clouds far from the origin."""
    w = inputs.make("slab", 1500, 24, T=10)
    off = np.array([500.0, -300.0, 250.0])
    q1, _, _ = gs.shoot(dt(w.q0 + off), dt(w.p0), w.sigma, w.T)
    q1o, _, _ = oracle.shoot(w.q0 + off, w.p0, w.sigma, w.T)
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma


def test_degenerate_clouds(oracle):
    """Coincident points and a flat (zero-thickness) cloud."""
    rng = np.random.default_rng(3)
    q = np.repeat(rng.normal(size=(1, 3)), 40, axis=0)
    p = rng.normal(scale=0.05, size=q.shape)
    q1, _, _ = gs.shoot(dt(q), dt(p), 1.0, 5)
    q1o, _, _ = oracle.shoot(q, p, 1.0, 5)
    assert np.abs(npy(q1) - q1o).max() <= 1e-5
    w = inputs.make("slab", 900, 25, T=5)
    q = w.q0.copy()
    q[:, 1] = 3.0
    q1, _, _ = gs.shoot(dt(q), dt(w.p0), w.sigma, w.T)
    q1o, _, _ = oracle.shoot(q, w.p0, w.sigma, w.T)
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma


def test_invalid_arguments_raise():
    w = inputs.make("slab", 10, 1)
    with pytest.raises(gs.GSError):
        gs.shoot(dt(w.q0), dt(w.p0), -1.0, 4)
    with pytest.raises(gs.GSError):
        gs.shoot(dt(w.q0), dt(w.p0), 1.0, 0)
    empty = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    for mode in ("exact", "bh"):
        with pytest.raises(gs.GSError) as ei:
            gs.shoot(empty, empty, 1.0, 4, mode=mode)
        assert ei.value.status == GS_ERR_INVALID_ARG
        with pytest.raises(gs.GSError) as ei:
            gs.shoot_grad(empty, empty, empty, 1.0, 4, mode=mode)
        assert ei.value.status == GS_ERR_INVALID_ARG
    with pytest.raises(gs.GSError):
        gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), 1.0, 4, lam=-1.0)
