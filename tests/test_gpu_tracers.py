"""Parity of the dense velocity field (Eq. 3) and of tracer points carried by
the shooting (gs_velocity, gs_flow) with the FP64 oracle, through the C ABI.

Tolerances as for the particles: positions max |dx(1)| <= 1e-5 sigma; one
field evaluation within 1e-5 of its own max."""
import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt, npy, max_rel

pytestmark = pytest.mark.gpu


def _tracers(w, m, seed, margin=4.0):
    """m points spread over the particles' box grown by `margin` sigma, plus
    a few far away (zero velocity)."""
    rng = np.random.default_rng(seed)
    lo = w.q0.min(0) - margin * w.sigma
    hi = w.q0.max(0) + margin * w.sigma
    x = lo + (hi - lo) * rng.random((m, 3))
    if m >= 4:
        x[:2] = w.q0.max(0) + 60.0 * w.sigma
    return x


@pytest.mark.parametrize("geom,n,m,seed", [("slab", 1, 1, 1), ("slab", 700, 255, 2),
                                          ("blobs", 2049, 257, 3), ("ellipsoid", 1000, 1000, 4),
                                          ("slab", 3000, 4097, 5)])
def test_velocity_matches_oracle(oracle, geom, n, m, seed):
    w = inputs.make(geom, n, seed)
    x = _tracers(w, m, seed)
    v = npy(gs.velocity(dt(w.q0), dt(w.p0), dt(x), w.sigma))
    vo = oracle.velocity(w.q0, w.p0, x, w.sigma)
    assert max_rel(v, vo) <= 1e-5
    if m >= 4:
        assert np.all(v[:2] == 0.0)


@pytest.mark.parametrize("geom,n,m,T", [("slab", 2000, 1500, 10), ("blobs", 1500, 600, 8),
                                        ("slab", 1, 3, 5)])
def test_flow_matches_oracle(oracle, geom, n, m, T):
    w = inputs.make(geom, n, 11 + n, T=T)
    x0 = _tracers(w, m, n)
    q1, p1, x1 = gs.flow(dt(w.q0), dt(w.p0), dt(x0), w.sigma, T)
    q1o, p1o, x1o = oracle.flow(w.q0, w.p0, x0, w.sigma, T)
    assert np.abs(npy(x1) - x1o).max() <= 1e-5 * w.sigma
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma
    assert max_rel(npy(p1), p1o) <= 1e-5


def test_tracers_on_particles_follow_them():
    w = inputs.make("slab", 1800, 21, T=12)
    x0 = w.q0[::5].copy()
    q1, _, x1 = gs.flow(dt(w.q0), dt(w.p0), dt(x0), w.sigma, w.T)
    assert np.abs(npy(x1) - npy(q1)[::5]).max() <= 1e-5 * w.sigma


def test_flow_without_tracers_equals_shoot():
    w = inputs.make("blobs", 900, 22, T=6)
    q1, p1, _ = gs.flow(dt(w.q0), dt(w.p0), torch.zeros((0, 3), dtype=torch.float64,
                                                        device="cuda"), w.sigma, w.T)
    q1s, p1s, _ = gs.shoot(dt(w.q0), dt(w.p0), w.sigma, w.T)
    assert torch.equal(q1, q1s) and torch.equal(p1, p1s)


def test_flow_graph_replay_bit_exact():
    w = inputs.make("slab", 1200, 23, T=7)
    x0 = dt(_tracers(w, 900, 23))
    q0, p0 = dt(w.q0), dt(w.p0)
    gs.set_option("graphs", 0)
    try:
        ref = gs.flow(q0, p0, x0, w.sigma, w.T)
    finally:
        gs.set_option("graphs", 1)
    for _ in range(2):
        got = gs.flow(q0, p0, x0, w.sigma, w.T)
        assert all(torch.equal(a, b) for a, b in zip(ref, got))


def test_flow_full_size_sampled(oracle):
    """N = 20,000 slab particles, 60,000 tracers on the slab's box, T = 20:
    tracers do not interact, so a sample of them is checked against the
    oracle run on that sample alone."""
    w = inputs.config("slab20k")
    x0 = _tracers(w, 60000, 31)
    _, _, x1 = gs.flow(dt(w.q0), dt(w.p0), dt(x0), w.sigma, w.T)
    rows = np.random.default_rng(5).choice(60000, 64, replace=False)
    _, _, x1o = oracle.flow(w.q0, w.p0, x0[rows], w.sigma, w.T)
    assert np.abs(npy(x1)[rows] - x1o).max() <= 1e-5 * w.sigma


def test_flow_rejects_truncation():
    w = inputs.make("slab", 10, 1)
    c = gs.context()
    from paper_1907_04834_gb300._lib import make_params
    import ctypes
    prm = make_params(w.sigma, 3, "trunc")
    q = dt(w.q0)
    out = torch.empty_like(q)
    st = c.lib.gs_flow(c.handle, ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(q.data_ptr()), 10,
                       ctypes.c_void_p(q.data_ptr()), 10, ctypes.byref(prm), None, None,
                       ctypes.c_void_p(out.data_ptr()), None)
    assert st == 6  # GS_ERR_UNSUPPORTED


@pytest.mark.parametrize("geom,n,m,seed,leaf,crit", [("blobs", 3000, 1000, 51, 1, 0),
                                                    ("slab", 2500, 777, 52, 1, 0),
                                                    ("sphere", 4000, 2049, 53, 8, 0),
                                                    ("blobs", 2000, 300, 54, 1, 1)])
def test_bh_velocity_matches_oracle(oracle, geom, n, m, seed, leaf, crit):
    """Barnes-Hut velocity at outside points (some beyond the particles' box,
    some far away): the same traversal decisions as the oracle's."""
    w = inputs.make(geom, n, seed)
    x = _tracers(w, m, seed)
    th = 0.6 if crit else 3.0
    v = npy(gs.velocity(dt(w.q0), dt(w.p0), dt(x), w.sigma, mode="bh", thresh=th, leaf_size=leaf,
                        criterion=crit))
    vo = oracle.velocity(w.q0, w.p0, x, w.sigma, mode=oracle.BH, thresh=th, leaf=leaf, crit=crit)
    assert max_rel(v, vo) <= 1e-5
    assert np.all(v[:2] == 0.0)


def test_bh_flow_matches_oracle(oracle):
    w = inputs.make("blobs", 2500, 55, T=8)
    x0 = _tracers(w, 1500, 55)
    q1, p1, x1 = gs.flow(dt(w.q0), dt(w.p0), dt(x0), w.sigma, w.T, mode="bh")
    q1o, p1o, x1o = oracle.flow(w.q0, w.p0, x0, w.sigma, w.T, mode=oracle.BH)
    assert np.abs(npy(x1) - x1o).max() <= 1e-5 * w.sigma
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma
    # Barnes-Hut tracers placed on particles follow them
    _, _, xp = gs.flow(dt(w.q0), dt(w.p0), dt(w.q0[::7]), w.sigma, w.T, mode="bh")
    assert np.abs(npy(xp) - npy(q1)[::7]).max() <= 1e-5 * w.sigma


def test_bh_flow_graph_replay_bit_exact():
    w = inputs.make("slab", 1500, 56, T=5)
    x0 = dt(_tracers(w, 1000, 56))
    q0, p0 = dt(w.q0), dt(w.p0)
    gs.set_option("graphs", 0)
    try:
        ref = gs.flow(q0, p0, x0, w.sigma, w.T, mode="bh")
    finally:
        gs.set_option("graphs", 1)
    for _ in range(2):
        got = gs.flow(q0, p0, x0, w.sigma, w.T, mode="bh")
        assert all(torch.equal(a, b) for a, b in zip(ref, got))


def test_bh_flow_full_size_sampled(oracle):
    """100,000 blob particles, 200,000 tracers, T = 4 (Barnes-Hut): a sample
    of tracers against the oracle run on that sample alone."""
    w = inputs.config("blobs100k")
    x0 = _tracers(w, 200000, 57)
    _, _, x1 = gs.flow(dt(w.q0), dt(w.p0), dt(x0), w.sigma, 4, mode="bh")
    rows = np.random.default_rng(6).choice(200000, 48, replace=False)
    _, _, x1o = oracle.flow(w.q0, w.p0, x0[rows], w.sigma, 4, mode=oracle.BH)
    assert np.abs(npy(x1)[rows] - x1o).max() <= 1e-5 * w.sigma
