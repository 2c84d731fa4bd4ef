"""gs_rhs and gs_adj_rhs walk the tree with the counting walk when counts are
asked for, and with the lean list walk of the paper's rule (the one every
shooting step uses) when they are not.  Both list the same entries in the
same order, so the right-hand sides are bit-identical; this pins the lean
walk's decisions to the counting walk's, whose totals the other tests hold
to the oracle's."""
import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt

pytestmark = pytest.mark.gpu


# one group, a group of one point after a full one, trees walked with two
# walk lists per slice, and a tree large enough for one (N >= 48 x SMs x 32)
@pytest.mark.parametrize("geom,n,seed", [("blobs", 1, 3), ("slab", 33, 4), ("blobs", 3000, 61),
                                         ("sphere", 5000, 6), ("blobs", 100000, 61),
                                         ("blobs", 250000, 61)])
def test_lean_walk_equals_counting_walk(geom, n, seed):
    w = inputs.make(geom, n, seed)
    rng = np.random.default_rng(seed)
    q, p = dt(w.q0), dt(w.p0)
    al, be = dt(rng.normal(size=w.q0.shape)), dt(rng.normal(scale=0.1, size=w.q0.shape))
    F, P, c = gs.rhs(q, p, w.sigma, mode="bh")
    F2, P2 = gs.rhs(q, p, w.sigma, mode="bh", with_counts=False)
    assert torch.equal(F, F2) and torch.equal(P, P2)
    A, B, ca = gs.adj_rhs(q, p, al, be, w.sigma, mode="bh")
    A2, B2 = gs.adj_rhs(q, p, al, be, w.sigma, mode="bh", with_counts=False)
    assert torch.equal(A, A2) and torch.equal(B, B2)
    assert tuple(c) == tuple(ca)
