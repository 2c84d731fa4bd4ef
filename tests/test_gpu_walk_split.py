"""The Barnes-Hut walk may cut each slice of a group's node range into two or
four walk lists (option bh_walk_split).  The evaluation reads a slice's walk lists
as one entry sequence in fixed batches, and a slice sent to the fused re-walk
(capped lists) is walked part after part with the lanes' state carried over,
so right-hand sides, adjoints, gradients, tracers and interaction counts are
bit-identical whichever split the walk used."""
import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt

pytestmark = pytest.mark.gpu


def _run_split(split, cap, fn):
    gs.set_option("bh_walk_split", split)
    gs.set_option("bh_list_cap", cap)
    try:
        return fn()
    finally:
        gs.set_option("bh_walk_split", 0)
        gs.set_option("bh_list_cap", 0)


CASES = [("blobs", 3000, 17, 0, "bh", 1), ("blobs", 3000, 17, 37, "bh", 1),
         ("blobs", 5000, 3, 1, "bh", 1), ("sphere", 5000, 6, 200, "bh", 1),
         ("slab", 777, 2, 0, "bh", 1), ("blobs", 4000, 9, 0, "bh", 8),
         ("blobs", 4000, 9, 23, "bh", 8), ("blobs", 3000, 5, 0, "trunc", 1),
         ("blobs", 3000, 5, 11, "trunc", 1)]


@pytest.mark.parametrize("geom,n,seed,cap,mode,leaf", CASES)
def test_walk_split_is_bit_exact(geom, n, seed, cap, mode, leaf):
    w = inputs.make(geom, n, seed, T=3)
    rng = np.random.default_rng(seed)
    al, be = dt(rng.normal(size=w.q0.shape)), dt(rng.normal(scale=0.1, size=w.q0.shape))
    kw = dict(mode=mode, leaf_size=leaf)

    def run():
        F, P, c = gs.rhs(dt(w.q0), dt(w.p0), w.sigma, **kw)
        A, B, ca = gs.adj_rhs(dt(w.q0), dt(w.p0), al, be, w.sigma, **kw)
        E, g, q1 = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam, **kw)
        return [F, P, A, B, E, g, q1], (tuple(c), tuple(ca))

    one, c1 = _run_split(1, cap, run)
    two, c2 = _run_split(2, cap, run)
    four, c4 = _run_split(4, cap, run)
    assert c1 == c2 == c4
    for a, b, c in zip(one, two, four):
        assert torch.equal(a, b) and torch.equal(a, c)


@pytest.mark.parametrize("cap", [0, 5])
def test_walk_split_tracers_bit_exact(cap):
    w = inputs.make("blobs", 2500, 44, T=4)
    rng = np.random.default_rng(4)
    x0 = w.q0[rng.choice(w.N, 700)] + rng.normal(scale=2.0, size=(700, 3))

    def run():
        return gs.flow(dt(w.q0), dt(w.p0), dt(x0), w.sigma, w.T, mode="bh")

    one = _run_split(1, cap, run)
    two = _run_split(2, cap, run)
    four = _run_split(4, cap, run)
    for a, b, c in zip(one, two, four):
        assert torch.equal(a, b) and torch.equal(a, c)


def test_walk_split_option_checked():
    with pytest.raises(Exception):
        gs.set_option("bh_walk_split", 3)
    with pytest.raises(Exception):
        gs.set_option("bh_walk_split", 8)
    gs.set_option("bh_walk_split", 0)


@pytest.mark.parametrize("cap", [0, 9])
def test_walk_split_forest_bit_exact(cap):
    """A forest of several subjects (batched Barnes-Hut) gives the same
    energies and gradients with one or two walk lists per slice."""
    specs = [("slab", 1200, 51), ("blobs", 700, 52), ("slab", 3, 53), ("ellipsoid", 513, 54)]
    ws = []
    for k, (g, n, seed) in enumerate(specs):
        w = inputs.make(g, n, seed, T=3, sigma=2.0)
        w.q0, w.X = w.q0 + 100.0 * k, w.X + 100.0 * k
        ws.append(w)
    q0 = np.concatenate([w.q0 for w in ws])
    p0 = np.concatenate([w.p0 for w in ws])
    X = np.concatenate([w.X for w in ws])
    off = np.cumsum([0] + [len(w.q0) for w in ws])

    def run():
        return gs.shoot_batched(dt(q0), dt(p0), dt(X), off, 2.0, 3, 1.0, mode="bh")

    one = _run_split(1, cap, run)
    two = _run_split(2, cap, run)
    four = _run_split(4, cap, run)
    for a, b, c in zip(one, two, four):
        assert torch.equal(a, b) and torch.equal(a, c)
