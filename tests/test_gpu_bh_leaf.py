"""Barnes-Hut leaf-size variant (gs_params.leaf_size > 1: a near node of at
most L points is taken exactly instead of opened) and the leaf-size
autotuner, against the oracle's same variant.  Interaction counts match the
oracle exactly; values to FP32 rounding; gradients within 1e-4."""
import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt, npy, max_rel, rel_l2, phi_floor

pytestmark = pytest.mark.gpu

CASES = [("blobs", 777, 3, 4), ("slab", 3000, 4, 8), ("blobs", 6000, 5, 16),
         ("sphere", 5000, 6, 32), ("blobs", 2, 7, 2)]


@pytest.mark.parametrize("geom,n,seed,leaf", CASES)
def test_leaf_rhs_matches_oracle(oracle, geom, n, seed, leaf):
    w = inputs.make(geom, max(n, 2), seed)
    q, p = w.q0[:n], w.p0[:n]
    F, Phi, cnt = gs.rhs(dt(q), dt(p), w.sigma, mode="bh", leaf_size=leaf)
    Fo, Phio, cnto = oracle.rhs(q, p, w.sigma, mode=1, leaf=leaf)
    assert tuple(cnt) == tuple(int(c) for c in cnto)
    assert max_rel(npy(F), Fo) <= 1e-5
    assert max_rel(npy(Phi), Phio, phi_floor(p, w.sigma)) <= 1e-5
    rng = np.random.default_rng(seed)
    al, be = rng.normal(size=q.shape), rng.normal(scale=0.1, size=q.shape)
    dA, dB, cnt = gs.adj_rhs(dt(q), dt(p), dt(al), dt(be), w.sigma, mode="bh", leaf_size=leaf)
    dAo, dBo, cnto = oracle.adj_rhs(q, p, al, be, w.sigma, mode=1, leaf=leaf)
    assert tuple(cnt) == tuple(int(c) for c in cnto)
    assert max_rel(npy(dA), dAo, 1e-12 * np.abs(al).max() * np.abs(p).max() / w.sigma) <= 1e-5
    assert max_rel(npy(dB), dBo) <= 1e-5


def test_leaf_gradient_matches_oracle(oracle):
    w = inputs.make("blobs", 2500, 8, T=6)
    E, g, q1 = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam, mode="bh",
                             leaf_size=8)
    Eo, go, q1o = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, w.lam, mode=1, leaf=8)
    assert rel_l2(npy(g), go) <= 1e-4
    np.testing.assert_allclose(npy(E), Eo, rtol=1e-6)
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma


@pytest.mark.parametrize("cap", [1, 8])
def test_leaf_list_overflow_is_bit_exact(cap):
    """Point entries survive the fused re-walk path bit for bit."""
    w = inputs.make("blobs", 3000, 9, T=3)
    args = (dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam)
    ref = gs.shoot_grad(*args, mode="bh", leaf_size=16)
    c0 = gs.rhs(dt(w.q0), dt(w.p0), w.sigma, mode="bh", leaf_size=16)[2]
    gs.set_option("bh_list_cap", cap)
    try:
        out = gs.shoot_grad(*args, mode="bh", leaf_size=16)
        c1 = gs.rhs(dt(w.q0), dt(w.p0), w.sigma, mode="bh", leaf_size=16)[2]
    finally:
        gs.set_option("bh_list_cap", 0)
    assert c0 == c1
    assert all(torch.equal(a, b) for a, b in zip(ref, out))


def test_leaf_forest_equals_single_sets():
    ws = [inputs.make("slab", n, 40 + n, T=3, sigma=2.0) for n in (900, 1, 1400)]
    off = np.zeros(4, np.int64)
    off[1:] = np.cumsum([w.N for w in ws])
    cat = lambda k: dt(np.concatenate([getattr(w, k) for w in ws]))
    E, g = gs.shoot_batched(cat("q0"), cat("p0"), cat("X"), off, 2.0, 3, 1.0, mode="bh",
                            leaf_size=8)
    for k, w in enumerate(ws):
        Ek, gk, _ = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), 2.0, 3, 1.0, mode="bh", leaf_size=8)
        assert torch.equal(E[k], Ek) and torch.equal(g[off[k]:off[k + 1]], gk), k


def test_leaf_size_one_is_the_paper_rule():
    w = inputs.make("blobs", 2000, 10, T=3)
    a = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam, mode="bh")
    b = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam, mode="bh", leaf_size=1)
    assert all(torch.equal(x, y) for x, y in zip(a, b))


def test_autotune_picks_a_candidate():
    w = inputs.make("blobs", 20000, 11)
    best, ms = gs.autotune(dt(w.q0), dt(w.p0), w.sigma)
    assert best in ms and all(v > 0 for v in ms.values())
    assert ms[best] == min(ms.values())
    print("\nleaf-size autotune, blobs N=20000:", best, {k: round(v, 3) for k, v in ms.items()})
    with pytest.raises(gs.GSError):
        gs.autotune(dt(w.q0), dt(w.p0), w.sigma, candidates=(0, 4))


@pytest.mark.parametrize("geom,n,seed,theta,leaf", [("blobs", 3000, 21, 0.5, 1),
                                                    ("sphere", 4000, 22, 0.8, 1),
                                                    ("slab", 2500, 23, 0.6, 8)])
def test_opening_angle_matches_oracle(oracle, geom, n, seed, theta, leaf):
    """Opening-angle variant (criterion 1): decisions equal the oracle's
    (interaction counts exact), values within FP32 rounding."""
    w = inputs.make(geom, n, seed)
    q, p = w.q0, w.p0
    F, Phi, cnt = gs.rhs(dt(q), dt(p), w.sigma, mode="bh", thresh=theta, leaf_size=leaf,
                         criterion=1)
    Fo, Phio, cnto = oracle.rhs(q, p, w.sigma, mode=1, thresh=theta, leaf=leaf, crit=1)
    assert tuple(cnt) == tuple(int(c) for c in cnto) and cnto[1] > 0
    assert max_rel(npy(F), Fo) <= 1e-5
    assert max_rel(npy(Phi), Phio, phi_floor(p, w.sigma)) <= 1e-5
    rng = np.random.default_rng(seed)
    al, be = rng.normal(size=q.shape), rng.normal(scale=0.1, size=q.shape)
    dA, dB, cnt = gs.adj_rhs(dt(q), dt(p), dt(al), dt(be), w.sigma, mode="bh", thresh=theta,
                             leaf_size=leaf, criterion=1)
    dAo, dBo, cnto = oracle.adj_rhs(q, p, al, be, w.sigma, mode=1, thresh=theta, leaf=leaf, crit=1)
    assert tuple(cnt) == tuple(int(c) for c in cnto)
    assert max_rel(npy(dA), dAo, 1e-12 * np.abs(al).max() * np.abs(p).max() / w.sigma) <= 1e-5
    assert max_rel(npy(dB), dBo) <= 1e-5


def test_opening_angle_gradient_and_overflow(oracle):
    w = inputs.make("blobs", 2000, 24, T=5)
    args = (dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam)
    E, g, q1 = gs.shoot_grad(*args, mode="bh", thresh=0.5, criterion=1)
    Eo, go, q1o = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, w.lam, mode=1, thresh=0.5,
                                    crit=1)
    assert rel_l2(npy(g), go) <= 1e-4
    np.testing.assert_allclose(npy(E), Eo, rtol=1e-6)
    gs.set_option("bh_list_cap", 2)
    try:
        E2, g2, q2 = gs.shoot_grad(*args, mode="bh", thresh=0.5, criterion=1)
    finally:
        gs.set_option("bh_list_cap", 0)
    assert torch.equal(E, E2) and torch.equal(g, g2) and torch.equal(q1, q2)


def test_opening_angle_argument_checks():
    w = inputs.make("blobs", 50, 25)
    with pytest.raises(gs.GSError):
        gs.rhs(dt(w.q0), dt(w.p0), w.sigma, mode="bh", thresh=3.0, criterion=1)  # theta > 1
    with pytest.raises(gs.GSError):
        gs.rhs(dt(w.q0), dt(w.p0), w.sigma, mode="trunc", thresh=0.5, criterion=1)
