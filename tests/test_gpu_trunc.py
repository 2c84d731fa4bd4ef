"""Pure 3-sigma truncation (GS_TRUNC, a variant compared with the paper's
Barnes-Hut approximation) against the oracle's plain double loop with the
same FP32 cutoff test: kept-pair counts equal exactly, values to FP32
rounding, gradients within 1e-4."""
import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt, npy, max_rel, rel_l2, phi_floor

pytestmark = pytest.mark.gpu

CASES = [("blobs", 1, 1, 3.0, 1), ("blobs", 777, 3, 3.0, 1), ("slab", 3000, 4, 2.0, 1),
         ("blobs", 5000, 5, 3.0, 16), ("sphere", 4000, 6, 3.0, 8), ("ellipsoid", 1000, 1001, 1.0, 1)]


@pytest.mark.parametrize("geom,n,seed,th,leaf", CASES)
def test_trunc_rhs_matches_oracle(oracle, geom, n, seed, th, leaf):
    w = inputs.make(geom, max(n, 2), seed)
    q, p = w.q0[:n], w.p0[:n]
    F, Phi, cnt = gs.rhs(dt(q), dt(p), w.sigma, mode="trunc", thresh=th, leaf_size=leaf)
    Fo, Phio, cnto = oracle.rhs(q, p, w.sigma, mode=oracle.TRUNC, thresh=th)
    assert tuple(cnt) == (int(cnto[0]), 0)
    assert max_rel(npy(F), Fo) <= 1e-5
    if n > 1:
        assert max_rel(npy(Phi), Phio, phi_floor(p, w.sigma)) <= 1e-5
    rng = np.random.default_rng(seed)
    al, be = rng.normal(size=q.shape), rng.normal(scale=0.1, size=q.shape)
    dA, dB, cnt = gs.adj_rhs(dt(q), dt(p), dt(al), dt(be), w.sigma, mode="trunc", thresh=th,
                             leaf_size=leaf)
    dAo, dBo, cnto = oracle.adj_rhs(q, p, al, be, w.sigma, mode=oracle.TRUNC, thresh=th)
    assert tuple(cnt) == (int(cnto[0]), 0)
    assert max_rel(npy(dA), dAo, 1e-12 * np.abs(al).max() * np.abs(p).max() / w.sigma) <= 1e-5
    assert max_rel(npy(dB), dBo) <= 1e-5


def test_trunc_gradient_matches_oracle(oracle):
    w = inputs.make("blobs", 2500, 8, T=6)
    E, g, q1 = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam, mode="trunc")
    Eo, go, q1o = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, w.lam, mode=oracle.TRUNC)
    assert rel_l2(npy(g), go) <= 1e-4
    np.testing.assert_allclose(npy(E), Eo, rtol=1e-6)
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma


@pytest.mark.parametrize("cap", [1, 8])
def test_trunc_list_overflow_is_bit_exact(cap):
    w = inputs.make("blobs", 3000, 9, T=3)
    args = (dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam)
    ref = gs.shoot_grad(*args, mode="trunc")
    c0 = gs.rhs(dt(w.q0), dt(w.p0), w.sigma, mode="trunc")[2]
    gs.set_option("bh_list_cap", cap)
    try:
        out = gs.shoot_grad(*args, mode="trunc")
        c1 = gs.rhs(dt(w.q0), dt(w.p0), w.sigma, mode="trunc")[2]
    finally:
        gs.set_option("bh_list_cap", 0)
    assert c0 == c1
    assert all(torch.equal(a, b) for a, b in zip(ref, out))


def test_trunc_forest_equals_single_sets():
    ws = [inputs.make("slab", n, 60 + n, T=3, sigma=2.0) for n in (800, 1, 1300)]
    off = np.zeros(4, np.int64)
    off[1:] = np.cumsum([w.N for w in ws])
    cat = lambda k: dt(np.concatenate([getattr(w, k) for w in ws]))
    E, g = gs.shoot_batched(cat("q0"), cat("p0"), cat("X"), off, 2.0, 3, 1.0, mode="trunc")
    for k, w in enumerate(ws):
        Ek, gk, _ = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), 2.0, 3, 1.0, mode="trunc")
        assert torch.equal(E[k], Ek) and torch.equal(g[off[k]:off[k + 1]], gk), k


def test_trunc_huge_threshold_is_exact():
    w = inputs.make("blobs", 2000, 10)
    F, Phi, cnt = gs.rhs(dt(w.q0), dt(w.p0), w.sigma, mode="trunc", thresh=1e4)
    Fe, Phie, _ = gs.rhs(dt(w.q0), dt(w.p0), w.sigma)
    assert cnt[0] == 2000 * 2000
    assert max_rel(npy(F), npy(Fe)) <= 1e-5
