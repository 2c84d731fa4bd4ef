"""The Barnes-Hut decisions and node statistics of the CUDA path against the
oracle, target by target and node by node (Sec. 2.2: the three cases of the
traversal, the node statistics n, sum q, sum p and the backward stage's
sum alpha, sum beta behind the summaries of Eq. 4).

Decisions: for every target, the number of points it takes exactly, the
number of nodes it summarises, a fingerprint of each set (a sum modulo
2^64 of a 64-bit mix of each source's identity) and the number of nodes the
traversal reaches must equal the oracle's bit for bit; a decision moved
from one target to another, or swapped between two sources of one target,
changes a record even where the totals stay equal.  Node statistics:
member counts exactly, sums within the rounding of their FP32 inputs (bound
computed per node from the members)."""
import numpy as np
import pytest

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt, npy
from test_gpu_tree import oracle_node_list

pytestmark = pytest.mark.gpu

CASES = [("blobs", 1, 1, 3.0, 1, 0), ("blobs", 2, 2, 3.0, 1, 0), ("blobs", 37, 3, 3.0, 1, 0),
         ("blobs", 4097, 5, 3.0, 1, 0), ("slab", 3000, 4, 3.0, 1, 0),
         ("ellipsoid", 1000, 1001, 2.0, 1, 0), ("sphere", 5000, 6, 3.0, 1, 0),
         ("blobs", 4000, 7, 1.0, 1, 0), ("blobs", 3000, 8, 3.0, 4, 0),
         ("slab", 2500, 9, 3.0, 32, 0), ("ellipsoid", 2000, 10, 0.6, 1, 1)]


def _cloud(geom, n, seed):
    w = inputs.make(geom, max(n, 2), seed)
    q = w.q0[:n].copy()
    if n >= 20:
        q[7] = q[3]           # exact duplicates: a depth-10 list
        q[8] = q[3]
        q[12] = q[11] + 1e-6  # same finest cell
    return w, q


def _as_u64(a):
    return np.ascontiguousarray(a).view(np.uint64)


@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("geom,n,seed,th,leaf,crit", CASES)
def test_decisions_per_target(oracle, geom, n, seed, th, leaf, crit, split):
    w, q = _cloud(geom, n, seed)
    gs.set_option("bh_walk_split", split)
    try:
        t = npy(gs.bh_tally(dt(q), w.sigma, th, leaf_size=leaf, criterion=crit))
    finally:
        gs.set_option("bh_walk_split", 0)
    to = oracle.bh_tally(q, w.sigma, th, leaf=leaf, crit=crit)
    bad = np.flatnonzero(np.any(t != to, axis=1))
    assert bad.size == 0, f"{bad.size} targets differ, first {bad[:5]}"
    # the walk of the right-hand side makes the same decisions in total
    _, _, cnt = gs.rhs(dt(q), dt(w.p0[:n]), w.sigma, mode="bh", thresh=th, leaf_size=leaf,
                       criterion=crit)
    assert tuple(cnt) == (int(t[:, 0].sum()), int(t[:, 1].sum()))


@pytest.mark.parametrize("name", ["blobs100k", "sphere1m"])
def test_decisions_per_target_full_size(oracle, name):
    """Every target's decisions at the benchmark's N = 100,000 and the largest
    workload's N = 1,000,000."""
    w = inputs.config(name)
    t, (iters, entries) = gs.bh_tally(dt(w.q0), w.sigma, with_stats=True)
    t = npy(t)
    to = oracle.bh_tally(w.q0, w.sigma)
    bad = np.flatnonzero(np.any(t != to, axis=1))
    visits = int(t[:, 0].sum() + t[:, 4].sum())
    taken = int(t[:, 0].sum() + t[:, 1].sum())
    print(f"\n{name}: {w.N} targets, {int(t[:, 0].sum())} point and {int(t[:, 1].sum())} node "
          f"interactions; targets whose decisions differ from the oracle's: {bad.size}; "
          f"traversal node visits {visits}, walk iterations {iters} ({visits / (32 * iters):.3f} "
          f"of their lane-slots), list entries {entries} ({taken / (32 * entries):.3f} of their "
          f"lane-slots taken)")
    assert bad.size == 0


def _oracle_stats(t):
    """Sums per stored node (the oracle's tree in the GPU's stored form:
    chains dropped, depth-10 lists expanded into their points)."""
    rows = []
    for k in range(len(t["depth"])):
        leaf, n, nch = int(t["leaf"][k]), int(t["n"][k]), int(t["nchild"][k])
        st = np.concatenate([t["sq"][k], t["sp"][k], t["sa"][k], t["sb"][k]])
        if not leaf:
            if nch >= 2:
                rows.append((int(t["first"][k]), n, st))
        elif n >= 2:
            rows.append((int(t["first"][k]), n, st))
            for pos in range(int(t["first"][k]), int(t["first"][k]) + n):
                rows.append((pos, 1, None))
        else:
            rows.append((int(t["first"][k]), 1, st))
    return rows


@pytest.mark.parametrize("geom,n,seed", [("blobs", 1, 1), ("blobs", 37, 3), ("slab", 3000, 4),
                                         ("blobs", 4097, 5), ("sphere", 5000, 6),
                                         ("ellipsoid", 2000, 7)])
def test_node_sums(oracle, geom, n, seed):
    w, q = _cloud(geom, n, seed)
    rng = np.random.default_rng(seed)
    p = w.p0[:n] if n > 1 else rng.normal(size=(1, 3))
    al = rng.normal(size=q.shape)
    be = rng.normal(scale=0.1, size=q.shape)
    S = npy(gs.tree_sums(dt(q), dt(p), dt(al), dt(be)))
    nodes = npy(gs.tree(dt(q))["nodes"]).astype(np.int64)
    t = oracle.tree(q, p, al, be)
    ref, _ = oracle_node_list(t)
    assert np.array_equal(nodes, ref)  # same nodes, same members
    rows = _oracle_stats(t)
    assert len(rows) == len(S)
    order = t["order"]
    # rounding bound of each sum: the GPU sums the FP32-rounded values
    # (positions relative to the bounding-box centre) with compensated
    # FP32 pairs; each input carries at most 2^-24 of its magnitude
    c = 0.5 * (q.min(axis=0) + q.max(axis=0))
    mag = np.concatenate([np.abs(q - c), np.abs(p), np.abs(al), np.abs(be)], axis=1)[order]
    cum = np.concatenate([np.zeros((1, 12)), np.cumsum(mag, axis=0)])
    worst = 0.0
    for e, (first, cnt, st) in enumerate(rows):
        assert (int(nodes[e, 1]), int(nodes[e, 2])) == (first, cnt)
        if st is None:  # a point of a depth-10 list: its own values
            i = order[first]
            st = np.concatenate([q[i], p[i], al[i], be[i]])
        bound = 2.0 ** -22 * (cum[first + cnt] - cum[first]) + 1e-300
        err = np.abs(S[e] - st)
        assert np.all(err <= bound), (e, err, bound)
        worst = max(worst, float((err / bound).max()))
    print(f"\n{geom} N={n}: {len(rows)} nodes, largest error / bound {worst:.3f}")
