"""Parity of the Barnes-Hut CUDA path (Sec. 2.2: octree, three-case
traversal, Eq. 4 summaries, backward-stage replacements) with the oracle's
Barnes-Hut.  On a shared state both sides take the same accept/open
decisions (FP32 rule), so interaction counts match exactly and values agree
to FP32 rounding; trajectories within 1e-5 sigma, gradients within 1e-4."""
import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt, npy, max_rel, rel_l2, phi_floor

pytestmark = pytest.mark.gpu

CASES = [("blobs", 1, 1, 3.0), ("blobs", 2, 2, 3.0), ("blobs", 777, 3, 3.0),
         ("slab", 3000, 4, 3.0), ("blobs", 4000, 5, 1.0), ("ellipsoid", 1000, 1001, 2.0),
         ("sphere", 5000, 6, 3.0)]


@pytest.mark.parametrize("geom,n,seed,th", CASES)
def test_bh_rhs_matches_oracle(oracle, geom, n, seed, th):
    w = inputs.make(geom, max(n, 2), seed)
    q, p = w.q0[:n], w.p0[:n]
    F, Phi, cnt = gs.rhs(dt(q), dt(p), w.sigma, mode="bh", thresh=th)
    Fo, Phio, cnto = oracle.rhs(q, p, w.sigma, mode=1, thresh=th)
    assert tuple(cnt) == tuple(int(c) for c in cnto)
    assert max_rel(npy(F), Fo) <= 1e-5
    if n > 1:
        assert max_rel(npy(Phi), Phio, phi_floor(p, w.sigma)) <= 1e-5


@pytest.mark.parametrize("geom,n,seed,th", CASES)
def test_bh_adjoint_rhs_matches_oracle(oracle, geom, n, seed, th):
    w = inputs.make(geom, max(n, 2), seed)
    q, p = w.q0[:n], w.p0[:n]
    rng = np.random.default_rng(seed)
    al, be = rng.normal(size=q.shape), rng.normal(scale=0.1, size=q.shape)
    dA, dB, cnt = gs.adj_rhs(dt(q), dt(p), dt(al), dt(be), w.sigma, mode="bh", thresh=th)
    dAo, dBo, cnto = oracle.adj_rhs(q, p, al, be, w.sigma, mode=1, thresh=th)
    assert tuple(cnt) == tuple(int(c) for c in cnto)
    assert max_rel(npy(dA), dAo, 1e-12 * np.abs(al).max() * np.abs(p).max() / w.sigma) <= 1e-5
    assert max_rel(npy(dB), dBo) <= 1e-5


@pytest.mark.parametrize("geom,n,seed,T,th", [("slab", 3000, 11, 20, 3.0),
                                              ("blobs", 2500, 12, 20, 3.0),
                                              ("ellipsoid", 1000, 1001, 10, 2.0)])
def test_bh_shoot_matches_oracle(oracle, geom, n, seed, T, th):
    w = inputs.make(geom, n, seed, T=T)
    q1, p1, H = gs.shoot(dt(w.q0), dt(w.p0), w.sigma, w.T, mode="bh", thresh=th, with_H=True)
    q1o, p1o, Ho = oracle.shoot(w.q0, w.p0, w.sigma, w.T, mode=1, thresh=th)
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma
    np.testing.assert_allclose(npy(H), Ho, rtol=1e-6)
    # the approximation's own error against exact shooting (reported)
    q1e, _, _ = oracle.shoot(w.q0, w.p0, w.sigma, w.T)
    print(f"\nBH vs exact {geom} N={n}: max|dq1|/sigma = {np.abs(q1o - q1e).max() / w.sigma:.3e}")


@pytest.mark.parametrize("geom,n,seed,T", [("slab", 2000, 13, 8), ("blobs", 1500, 14, 6)])
def test_bh_gradient_matches_oracle(oracle, geom, n, seed, T):
    w = inputs.make(geom, n, seed, T=T)
    E, g, q1 = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam, mode="bh")
    Eo, go, q1o = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, w.lam, mode=1)
    assert rel_l2(npy(g), go) <= 1e-4
    np.testing.assert_allclose(npy(E), Eo, rtol=1e-6)
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma
    _, ge, _ = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, w.lam)
    print(f"\nBH grad vs exact grad {geom} N={n}: rel L2 = {rel_l2(go, ge):.3e}")


def test_bh_checkpointing_is_bit_exact():
    w = inputs.make("blobs", 2000, 15, T=9)
    a = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam, mode="bh")
    b = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam, mode="bh", ckpt_every=4)
    for x, y in zip(a, b):
        assert np.array_equal(npy(x), npy(y))


def test_infinite_threshold_equals_exact():
    w = inputs.make("blobs", 3000, 16)
    F, Phi, cnt = gs.rhs(dt(w.q0), dt(w.p0), w.sigma, mode="bh", thresh=1e30)
    Fe, Phie, _ = gs.rhs(dt(w.q0), dt(w.p0), w.sigma)
    assert cnt == (3000 * 3000, 0)
    assert max_rel(npy(F), npy(Fe)) <= 1e-5
    assert max_rel(npy(Phi), npy(Phie)) <= 1e-5


def test_bh_fullsize_single_step(oracle):
    """N = 100,000 blobs at sigma = 1.5: one Barnes-Hut forward and one
    backward right-hand side against the full oracle, identical decisions."""
    w = inputs.config("blobs100k")
    F, Phi, cnt = gs.rhs(dt(w.q0), dt(w.p0), w.sigma, mode="bh")
    Fo, Phio, cnto = oracle.rhs(w.q0, w.p0, w.sigma, mode=1)
    assert tuple(cnt) == tuple(int(c) for c in cnto)
    assert max_rel(npy(F), Fo) <= 1e-5 and max_rel(npy(Phi), Phio) <= 1e-5
    rng = np.random.default_rng(1)
    al, be = rng.normal(size=w.q0.shape), rng.normal(scale=0.1, size=w.q0.shape)
    dA, dB, cnt = gs.adj_rhs(dt(w.q0), dt(w.p0), dt(al), dt(be), w.sigma, mode="bh")
    dAo, dBo, cnto = oracle.adj_rhs(w.q0, w.p0, al, be, w.sigma, mode=1)
    assert tuple(cnt) == tuple(int(c) for c in cnto)
    assert max_rel(npy(dA), dAo) <= 1e-5 and max_rel(npy(dB), dBo) <= 1e-5
    print(f"\nN=100k BH interactions per point: {cnt[0] / w.N:.0f} point + {cnt[1] / w.N:.0f} node")


@pytest.mark.parametrize("cap", [1, 37, 200])
def test_list_overflow_is_bit_exact(cap):
    """Lists capped far below their length send slices to the fused
    walk-and-evaluate pass, which batches exactly like the list evaluation:
    results and interaction counts are bit-identical to uncapped lists."""
    w = inputs.make("blobs", 3000, 17, T=3)
    args = (dt(w.q0), dt(w.p0), w.sigma)
    rng = np.random.default_rng(0)
    al, be = dt(rng.normal(size=w.q0.shape)), dt(rng.normal(size=w.q0.shape))

    def run():
        F, P, c = gs.rhs(*args, mode="bh")
        A, B, _ = gs.adj_rhs(dt(w.q0), dt(w.p0), al, be, w.sigma, mode="bh")
        E, g, q1 = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam, mode="bh")
        return [F, P, A, B, E, g, q1], c

    ref, c0 = run()
    gs.set_option("bh_list_cap", cap)
    try:
        out, c1 = run()
    finally:
        gs.set_option("bh_list_cap", 0)
    assert c1 == c0
    for a, b in zip(out, ref):
        assert torch.equal(a, b)


def _degenerate(kind):
    rng = np.random.default_rng(71)
    if kind == "cluster":  # 300 coincident points (one depth-10 cell) among 400 others
        q = np.vstack([np.repeat(rng.normal(size=(1, 3)), 300, axis=0),
                       rng.normal(scale=4.0, size=(400, 3))])
    elif kind == "flat":  # a zero-extent axis: every z equal
        q = rng.normal(scale=5.0, size=(900, 3))
        q[:, 2] = 1.25
    elif kind == "line":  # collinear points
        t = rng.uniform(-20, 20, size=(600, 1))
        q = t * np.array([[0.6, -0.48, 0.64]]) + np.array([[1.0, 2.0, 3.0]])
    else:  # every point at the same position
        q = np.repeat(np.array([[3.0, -1.0, 2.0]]), 64, axis=0)
    p = rng.normal(scale=0.1, size=q.shape)
    return q, p


@pytest.mark.parametrize("kind", ["cluster", "flat", "line", "all_same"])
def test_bh_degenerate_clouds(oracle, kind):
    q, p = _degenerate(kind)
    sigma = 1.0
    F, Phi, cnt = gs.rhs(dt(q), dt(p), sigma, mode="bh")
    Fo, Phio, cnto = oracle.rhs(q, p, sigma, mode=1)
    assert tuple(cnt) == tuple(int(c) for c in cnto)
    assert max_rel(npy(F), Fo) <= 1e-5
    assert max_rel(npy(Phi), Phio, phi_floor(p, sigma)) <= 1e-5
    rng = np.random.default_rng(3)
    al, be = rng.normal(size=q.shape), rng.normal(scale=0.1, size=q.shape)
    dA, dB, cnt = gs.adj_rhs(dt(q), dt(p), dt(al), dt(be), sigma, mode="bh")
    dAo, dBo, cnto = oracle.adj_rhs(q, p, al, be, sigma, mode=1)
    assert tuple(cnt) == tuple(int(c) for c in cnto)
    assert max_rel(npy(dA), dAo, 1e-12 * np.abs(al).max() * np.abs(p).max() / sigma) <= 1e-5
    assert max_rel(npy(dB), dBo) <= 1e-5
