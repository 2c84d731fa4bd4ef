"""Pure truncation over a uniform cell grid (option trunc_grid of GS_TRUNC):
the same pairs as the oracle's plain double loop with the FP32 cutoff test
(kept-pair counts equal exactly, values to FP32 rounding), the same counts
as the octree search, and bit-identical reruns and graph replays."""
import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt, npy, max_rel, rel_l2, phi_floor

pytestmark = pytest.mark.gpu


def _grid(fn):
    gs.set_option("trunc_grid", 1)
    try:
        return fn()
    finally:
        gs.set_option("trunc_grid", 0)


def _clouds():
    rng = np.random.default_rng(0)
    out = []
    for geom, n, seed, th in [("blobs", 1, 1, 3.0), ("blobs", 2, 2, 3.0), ("blobs", 777, 3, 3.0),
                              ("slab", 3000, 4, 2.0), ("sphere", 4000, 6, 3.0),
                              ("ellipsoid", 1000, 1001, 1.0)]:
        w = inputs.make(geom, max(n, 2), seed)
        out.append((f"{geom}{n}", w.q0[:n], w.p0[:n], w.sigma, th))
    flat = rng.normal(size=(500, 3)) * 3.0
    flat[:, 2] = 1.25  # one cell along z
    out.append(("flat_z", flat, rng.normal(scale=0.1, size=(500, 3)), 1.0, 3.0))
    out.append(("coincident", np.repeat(rng.normal(size=(5, 3)), 40, axis=0),
                rng.normal(scale=0.1, size=(200, 3)), 0.5, 3.0))
    # 200 points in a 40-sigma cube: 26^3 cells of side 1.53 sigma exceed the
    # cap of 8 N + 4096, so the cell side is doubled
    sparse = rng.uniform(-20.0, 20.0, size=(200, 3))
    out.append(("sparse_cube", sparse, rng.normal(scale=0.1, size=(200, 3)), 1.0, 3.0))
    return [pytest.param(*c, id=c[0]) for c in out]


@pytest.mark.parametrize("name,q,p,sigma,th", _clouds())
def test_grid_rhs_matches_oracle(oracle, name, q, p, sigma, th):
    F, Phi, cnt = _grid(lambda: gs.rhs(dt(q), dt(p), sigma, mode="trunc", thresh=th))
    Fo, Phio, cnto = oracle.rhs(q, p, sigma, mode=oracle.TRUNC, thresh=th)
    assert tuple(cnt) == (int(cnto[0]), 0)
    assert max_rel(npy(F), Fo) <= 1e-5
    if len(q) > 1:
        assert max_rel(npy(Phi), Phio, phi_floor(p, sigma)) <= 1e-5
    rng = np.random.default_rng(len(q))
    al, be = rng.normal(size=q.shape), rng.normal(scale=0.1, size=q.shape)
    dA, dB, cnt = _grid(lambda: gs.adj_rhs(dt(q), dt(p), dt(al), dt(be), sigma, mode="trunc",
                                           thresh=th))
    dAo, dBo, cnto = oracle.adj_rhs(q, p, al, be, sigma, mode=oracle.TRUNC, thresh=th)
    assert tuple(cnt) == (int(cnto[0]), 0)
    assert max_rel(npy(dA), dAo, 1e-12 * np.abs(al).max() * np.abs(p).max() / sigma) <= 1e-5
    assert max_rel(npy(dB), dBo) <= 1e-5


def test_grid_gradient_matches_oracle(oracle):
    w = inputs.make("blobs", 2500, 8, T=6)
    E, g, q1 = _grid(lambda: gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam,
                                           mode="trunc"))
    Eo, go, q1o = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, w.lam, mode=oracle.TRUNC)
    assert rel_l2(npy(g), go) <= 1e-4
    np.testing.assert_allclose(npy(E), Eo, rtol=1e-6)
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma


def test_grid_equals_octree_search():
    """Both searches keep the same pairs; only the summation order differs."""
    w = inputs.make("blobs", 5000, 5, T=4)
    octree = gs.rhs(dt(w.q0), dt(w.p0), w.sigma, mode="trunc")
    grid = _grid(lambda: gs.rhs(dt(w.q0), dt(w.p0), w.sigma, mode="trunc"))
    assert tuple(grid[2]) == tuple(octree[2])
    assert max_rel(npy(grid[0]), npy(octree[0])) <= 1e-6
    args = (dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam)
    go = gs.shoot_grad(*args, mode="trunc")[1]
    gg = _grid(lambda: gs.shoot_grad(*args, mode="trunc"))[1]
    assert rel_l2(npy(gg), npy(go)) <= 1e-6


def test_grid_reruns_graphs_and_checkpoints_bit_exact():
    w = inputs.make("slab", 2000, 7, T=5)
    args = (dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam)
    a = _grid(lambda: gs.shoot_grad(*args, mode="trunc"))
    b = _grid(lambda: gs.shoot_grad(*args, mode="trunc"))
    c = _grid(lambda: gs.shoot_grad(*args, mode="trunc", ckpt_every=2))
    gs.set_option("graphs", 0)
    try:
        d = _grid(lambda: gs.shoot_grad(*args, mode="trunc"))
    finally:
        gs.set_option("graphs", 1)
    for x in (b, c, d):
        for u, v in zip(a, x):
            assert torch.equal(u, v)


def test_grid_option_checked():
    with pytest.raises(gs.GSError):
        gs.set_option("trunc_grid", 2)
    gs.set_option("trunc_grid", 0)
