"""The GPU octree against the oracle's insertion octree (Sec. 2.2), bit for
bit: Morton codes, the depth-first point order, the node list (cells with
>= 2 non-empty children, depth-10 groups, single-point leaves) with each
node's first member, size and subtree end, and each node's FP32 range."""
import numpy as np
import pytest

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt, npy

pytestmark = pytest.mark.gpu


def oracle_node_list(t):
    """The oracle's tree reduced to the stored form: drop single-child chain
    cells (same members and range as their child), expand depth-10 groups
    into one node followed by its points, and compute subtree ends."""
    seq = []
    for k in range(len(t["depth"])):
        d, leaf, n, first, nch = (int(t["depth"][k]), int(t["leaf"][k]), int(t["n"][k]),
                                  int(t["first"][k]), int(t["nchild"][k]))
        lohi = np.concatenate([t["lo"][k], t["hi"][k]])
        if not leaf:
            if nch >= 2:
                seq.append([d, first, n, lohi])
        elif n >= 2:
            seq.append([d, first, n, lohi])
            for pos in range(first, first + n):
                seq.append([-1, pos, 1, None])
        else:
            seq.append([-1, first, 1, lohi])
    out = np.zeros((len(seq), 4), np.int64)
    for e, (d, first, n, _) in enumerate(seq):
        end = e + 1
        while end < len(seq) and seq[end][1] < first + n:
            end += 1
        out[e] = (d, first, n, end)
    return out, seq


@pytest.mark.parametrize("geom,n,seed", [("blobs", 1, 1), ("blobs", 2, 2), ("blobs", 37, 3),
                                         ("slab", 1000, 4), ("blobs", 4097, 5),
                                         ("ellipsoid", 3000, 6)])
def test_tree_bit_exact(oracle, geom, n, seed):
    w = inputs.make(geom, max(n, 2), seed)
    q = w.q0[:n].copy()
    if n >= 20:
        q[7] = q[3]            # exact duplicates -> depth-10 group
        q[8] = q[3]
        q[12] = q[11] + 1e-6   # same finest cell
    g = gs.tree(dt(q))
    kq, code = oracle.morton(q)
    assert np.array_equal(npy(g["codes"]).view(np.uint32), code)
    t = oracle.tree(q, np.zeros_like(q))
    assert np.array_equal(npy(g["order"]).astype(np.int64), t["order"])
    ref, seq = oracle_node_list(t)
    nodes = npy(g["nodes"]).astype(np.int64)
    assert g["n_nodes"] == len(ref)
    assert np.array_equal(nodes, ref)
    rng = npy(g["range"])
    q32 = q.astype(np.float32)
    order = t["order"]
    for e, (d, first, cnt, lohi) in enumerate(seq):
        want = lohi if lohi is not None else np.concatenate([q32[order[first]]] * 2)
        assert np.array_equal(rng[e], want.astype(np.float32)), e


def test_tree_flat_axis(oracle):
    w = inputs.make("slab", 500, 9)
    q = w.q0.copy()
    q[:, 2] = 1.5
    g = gs.tree(dt(q))
    _, code = oracle.morton(q)
    assert np.array_equal(npy(g["codes"]).view(np.uint32), code)
    t = oracle.tree(q, np.zeros_like(q))
    ref, _ = oracle_node_list(t)
    assert np.array_equal(npy(g["nodes"]).astype(np.int64), ref)


@pytest.mark.parametrize("n,distinct,seed", [(9000, 7, 21), (70000, 3000, 22), (5000, 1, 23)])
def test_tree_heavy_duplicates(oracle, n, distinct, seed):
    """Many equal codes spread over many sort tiles: the sort must keep
    equal codes in input order (the oracle's insertion order), whole
    depth-10 lists included."""
    w = inputs.make("blobs", distinct + 1, seed)
    rng = np.random.default_rng(seed)
    q = w.q0[rng.integers(0, distinct, size=n)].copy() if distinct > 1 else \
        np.repeat(w.q0[:1], n, axis=0)
    g = gs.tree(dt(q))
    _, code = oracle.morton(q)
    assert np.array_equal(npy(g["codes"]).view(np.uint32), code)
    t = oracle.tree(q, np.zeros_like(q))
    assert np.array_equal(npy(g["order"]).astype(np.int64), t["order"])
    ref, _ = oracle_node_list(t)
    assert np.array_equal(npy(g["nodes"]).astype(np.int64), ref)
