"""Pins for the oracle's Barnes-Hut part (Sec. 2.2): the insertion octree
against brute-force cell enumeration, the traversal's interaction lists
against the three-case rule, and the summaries against cases where the
approximation is exact."""
import numpy as np
import pytest

from paper_1907_04834_gb300 import inputs


def _quantise_f32(q):
    """The quantisation rule written directly in numpy float32 (each op rounds to FP32)."""
    q32 = q.astype(np.float32)
    lo, hi = q32.min(axis=0), q32.max(axis=0)
    ext = hi - lo
    k = np.zeros(q.shape, np.uint32)
    for a in range(3):
        if ext[a] > 0:
            inv = np.float32(1024.0) / ext[a]
            u = (q32[:, a] - lo[a]) * inv
            k[:, a] = np.minimum(u.astype(np.uint32), 1023)
    return k


def _interleave(k):
    code = np.zeros(len(k), np.uint64)
    for b in range(10):
        code |= ((k[:, 0].astype(np.uint64) >> b) & 1) << (3 * b + 2)
        code |= ((k[:, 1].astype(np.uint64) >> b) & 1) << (3 * b + 1)
        code |= ((k[:, 2].astype(np.uint64) >> b) & 1) << (3 * b)
    return code


def _cloud_with_duplicates(n, seed):
    w = inputs.make("blobs", n, seed)
    q = w.q0.copy()
    q[5] = q[4]            # exact duplicates end in a finest-cell list
    q[9] = q[4]
    q[11] = q[10] + 1e-7   # same finest cell, different position
    return q, w.p0


def test_quantisation_and_morton(oracle):
    q, _ = _cloud_with_duplicates(500, 1)
    kq, code = oracle.morton(q)
    kb = _quantise_f32(q)
    assert np.array_equal(kq, kb)
    assert kq.min() == 0 and kq.max() == 1023
    lo_pts = np.argmin(q.astype(np.float32), axis=0)
    hi_pts = np.argmax(q.astype(np.float32), axis=0)
    for a in range(3):
        assert kq[lo_pts[a], a] == 0 and kq[hi_pts[a], a] == 1023
    assert np.array_equal(code.astype(np.uint64), _interleave(kq))
    # a flat axis (zero extent) quantises to 0
    qf = q.copy()
    qf[:, 2] = 4.25
    kf, _ = oracle.morton(qf)
    assert np.all(kf[:, 2] == 0)


@pytest.mark.parametrize("n,seed", [(2, 0), (37, 1), (300, 2), (1000, 3)])
def test_tree_matches_bruteforce_cells(oracle, n, seed):
    q, p = _cloud_with_duplicates(max(n, 12), seed)
    q, p = q[:n], p[:n]
    rng = np.random.default_rng(seed)
    al, be = rng.normal(size=q.shape), rng.normal(size=q.shape)
    t = oracle.tree(q, p, al, be)
    code = _interleave(_quantise_f32(q))
    # DFS point order = stable Morton order
    assert np.array_equal(t["order"], np.argsort(code, kind="stable"))
    # brute force: the cell of depth D exists iff D = 0 or its parent cell
    # holds >= 2 points (an occupied leaf is split when a second point arrives)
    cells = {}
    for D in range(11):
        pref = code >> np.uint64(30 - 3 * D)
        for c in np.unique(pref):
            mem = np.nonzero(pref == c)[0]
            cells[(D, int(c))] = mem
    exist = {key for key in cells if key[0] == 0 or
             len(cells[(key[0] - 1, key[1] >> 3)]) >= 2}
    assert len(t["depth"]) == len(exist)
    q32 = q.astype(np.float32)
    for k in range(len(t["depth"])):
        D, first, cnt = int(t["depth"][k]), int(t["first"][k]), int(t["n"][k])
        mem = np.sort(t["order"][first:first + cnt])
        c = int(code[mem[0]] >> np.uint64(30 - 3 * D))
        assert (D, c) in exist
        assert np.array_equal(mem, np.sort(cells[(D, c)]))
        assert t["leaf"][k] == int(cnt == 1 or D == 10)
        nch = sum(1 for o in range(8) if (D + 1, 8 * c + o) in exist) if D < 10 else 0
        assert t["nchild"][k] == (0 if t["leaf"][k] else nch)
        np.testing.assert_allclose(t["sq"][k], q[mem].sum(axis=0), rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(t["sp"][k], p[mem].sum(axis=0), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(t["sa"][k], al[mem].sum(axis=0), rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(t["sb"][k], be[mem].sum(axis=0), rtol=1e-13, atol=1e-12)
        assert np.array_equal(t["lo"][k], q32[mem].min(axis=0))
        assert np.array_equal(t["hi"][k], q32[mem].max(axis=0))


def _far(x32, lo, hi, thr):
    d = np.maximum(np.maximum(lo - x32, np.float32(0)), x32 - hi).astype(np.float32)
    d2 = np.float32(d[0] * d[0])
    d2 = np.float32(d2 + np.float32(d[1] * d[1]))
    d2 = np.float32(d2 + np.float32(d[2] * d[2]))
    return bool(d2 > thr)


@pytest.mark.parametrize("geom,n,thresh", [("blobs", 250, 3.0), ("slab", 300, 3.0),
                                           ("blobs", 200, 1.0)])
def test_interaction_lists_follow_three_cases(oracle, geom, n, thresh):
    """For each target: the sources partition all points exactly once; every
    summarised node has n >= 2 and is far; its parent is not far; every point
    taken exactly sits in a leaf whose ancestors are all not far."""
    w = inputs.make(geom, n, 17)
    q, p = w.q0, w.p0
    sigma = w.sigma * 0.6
    t = oracle.tree(q, p)
    r = np.float32(thresh * sigma)
    thr = np.float32(r * r)
    q32 = q.astype(np.float32)
    pos = np.empty(n, np.int64)
    pos[t["order"]] = np.arange(n)
    # leaf node of each point
    leaf_of = np.empty(n, np.int64)
    for k in np.nonzero(t["leaf"])[0]:
        leaf_of[t["order"][t["first"][k]:t["first"][k] + t["n"][k]]] = k
    n_far_total = 0
    for m in range(0, n, 7):
        kind, ids = oracle.bh_list(q, p, sigma, m, thresh)
        seen = np.zeros(n, np.int64)
        for kd, i in zip(kind, ids):
            if kd == 1:
                n_far_total += 1
                assert t["n"][i] >= 2
                assert _far(q32[m], t["lo"][i], t["hi"][i], thr)
                par = t["parent"][i]
                if par >= 0:
                    assert not _far(q32[m], t["lo"][par], t["hi"][par], thr)
                seen[t["order"][t["first"][i]:t["first"][i] + t["n"][i]]] += 1
            else:
                seen[i] += 1
                k = leaf_of[i]
                if t["n"][k] >= 2:
                    assert not _far(q32[m], t["lo"][k], t["hi"][k], thr)
                a = t["parent"][k]
                while a >= 0:
                    assert not _far(q32[m], t["lo"][a], t["hi"][a], thr)
                    a = t["parent"][a]
        assert np.all(seen == 1)
    assert n_far_total > 0  # the case actually exercises summaries


def test_infinite_threshold_is_exact(oracle):
    w = inputs.make("blobs", 400, 5, T=3)
    F, Phi, c0 = oracle.rhs(w.q0, w.p0, w.sigma)
    Fb, Phib, cb = oracle.rhs(w.q0, w.p0, w.sigma, mode=1, thresh=1e30)
    assert cb[1] == 0 and cb[0] == 400 * 400
    np.testing.assert_allclose(Fb, F, rtol=1e-12, atol=1e-15 * np.abs(F).max())
    np.testing.assert_allclose(Phib, Phi, rtol=1e-12, atol=1e-13 * np.abs(Phi).max())
    rng = np.random.default_rng(0)
    al, be = rng.normal(size=w.q0.shape), rng.normal(size=w.q0.shape)
    dA, dB, _ = oracle.adj_rhs(w.q0, w.p0, al, be, w.sigma)
    dAb, dBb, _ = oracle.adj_rhs(w.q0, w.p0, al, be, w.sigma, mode=1, thresh=1e30)
    np.testing.assert_allclose(dAb, dA, rtol=1e-11, atol=1e-13 * np.abs(dA).max())
    np.testing.assert_allclose(dBb, dB, rtol=1e-11, atol=1e-13 * np.abs(dB).max())
    E, g, q1 = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, 1.0)
    Eb, gb, q1b = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, 1.0, mode=1, thresh=1e30)
    np.testing.assert_allclose(q1b, q1, rtol=0, atol=1e-12)
    np.testing.assert_allclose(gb, g, rtol=1e-10, atol=1e-12 * np.abs(g).max())


def _cluster_case(identical):
    rng = np.random.default_rng(3)
    sigma = 1.0
    near = rng.uniform(-0.5, 0.5, size=(30, 3))
    c = np.array([6.0, 0.5, -0.25])
    far = np.repeat(c[None, :], 25, axis=0)
    pn = rng.normal(scale=0.3, size=(30, 3))
    pf = np.repeat(np.array([[0.2, -0.1, 0.4]]), 25, axis=0)
    an, bn = rng.normal(size=(30, 3)), rng.normal(size=(30, 3))
    af = np.repeat(np.array([[0.3, 0.7, -0.2]]), 25, axis=0)
    bf = np.repeat(np.array([[-0.5, 0.1, 0.9]]), 25, axis=0)
    if not identical:
        far = far + rng.normal(scale=0.3, size=far.shape)
        pf = pf + rng.normal(scale=0.3, size=pf.shape)
    q = np.vstack([near, far])
    return q, np.vstack([pn, pf]), np.vstack([an, af]), np.vstack([bn, bf]), sigma


def test_coincident_far_cluster_summary_is_exact(oracle):
    """A far cluster of n coincident points with equal p, alpha, beta is
    represented exactly by its summary (centroid, P, A, B/n): the replacement
    rules after Eq. 4 carry the multiplicity n, so forward and backward
    Barnes-Hut sums equal the exact sums for the other points."""
    q, p, al, be, sigma = _cluster_case(True)
    F, Phi, _ = oracle.rhs(q, p, sigma)
    Fb, Phib, cnt = oracle.rhs(q, p, sigma, mode=1, thresh=3.0)
    assert cnt[1] >= 30
    np.testing.assert_allclose(Fb[:30], F[:30], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Phib[:30], Phi[:30], rtol=1e-12, atol=1e-15)
    dA, dB, _ = oracle.adj_rhs(q, p, al, be, sigma)
    dAb, dBb, _ = oracle.adj_rhs(q, p, al, be, sigma, mode=1, thresh=3.0)
    np.testing.assert_allclose(dAb[:30], dA[:30], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(dBb[:30], dB[:30], rtol=1e-12, atol=1e-14)
    # control: a spread-out cluster is only approximated
    q, p, al, be, sigma = _cluster_case(False)
    F, _, _ = oracle.rhs(q, p, sigma)
    Fb, _, _ = oracle.rhs(q, p, sigma, mode=1, thresh=3.0)
    assert np.abs(Fb[:30] - F[:30]).max() > 1e-8


def test_bh_error_shrinks_with_threshold(oracle):
    w = inputs.make("blobs", 1500, 6)
    F, Phi, _ = oracle.rhs(w.q0, w.p0, w.sigma)
    errs = []
    for th in (2.0, 3.0, 4.0, 5.0):
        Fb, _, _ = oracle.rhs(w.q0, w.p0, w.sigma, mode=1, thresh=th)
        errs.append(np.abs(Fb - F).max() / np.abs(F).max())
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[1] < 1e-2


@pytest.mark.parametrize("leaf", [4, 16])
def test_leaf_size_variant_lists(oracle, leaf):
    """Leaf-size variant: a near node of at most `leaf` points is taken
    exactly instead of opened.  Sources still partition all points; a
    summarised node is far, and every ancestor is near and holds more than
    `leaf` points; the summaries are a subset of the paper's (leaf = 1)."""
    n = 260
    w = inputs.make("blobs", n, 23)
    q, p = w.q0, w.p0
    sigma = w.sigma * 0.6
    t = oracle.tree(q, p)
    r = np.float32(3.0 * sigma)
    thr = np.float32(r * r)
    q32 = q.astype(np.float32)
    fewer = 0
    for m in range(0, n, 5):
        kind, ids = oracle.bh_list(q, p, sigma, m, 3.0, leaf=leaf)
        kind1, ids1 = oracle.bh_list(q, p, sigma, m, 3.0)
        seen = np.zeros(n, np.int64)
        for kd, i in zip(kind, ids):
            if kd == 1:
                assert _far(q32[m], t["lo"][i], t["hi"][i], thr)
                a = t["parent"][i]
                while a >= 0:
                    assert not _far(q32[m], t["lo"][a], t["hi"][a], thr)
                    assert t["n"][a] > leaf
                    a = t["parent"][a]
                seen[t["order"][t["first"][i]:t["first"][i] + t["n"][i]]] += 1
            else:
                seen[i] += 1
        assert np.all(seen == 1)
        far_l = set(ids[kind == 1].tolist())
        far_1 = set(ids1[kind1 == 1].tolist())
        assert far_l <= far_1
        fewer += len(far_1) - len(far_l)
    assert fewer > 0  # the variant changes something here


def test_leaf_size_limits(oracle):
    """leaf = 1 is the paper's rule, bit for bit; leaf >= N takes every pair
    exactly (the root holds the target, so it is never far)."""
    w = inputs.make("blobs", 300, 29, T=3)
    F1, P1, c1 = oracle.rhs(w.q0, w.p0, w.sigma, mode=1)
    Fl, Pl, cl = oracle.rhs(w.q0, w.p0, w.sigma, mode=1, leaf=1)
    assert np.array_equal(F1, Fl) and np.array_equal(P1, Pl) and np.array_equal(c1, cl)
    Fe, Pe, _ = oracle.rhs(w.q0, w.p0, w.sigma)
    FN, PN, cN = oracle.rhs(w.q0, w.p0, w.sigma, mode=1, leaf=300)
    assert cN[0] == 300 * 300 and cN[1] == 0
    np.testing.assert_allclose(FN, Fe, rtol=1e-12, atol=1e-15 * np.abs(Fe).max())
    np.testing.assert_allclose(PN, Pe, rtol=1e-12, atol=1e-13 * np.abs(Pe).max())
    # interactions move from node summaries to exact pairs as leaf grows
    c4 = oracle.rhs(w.q0, w.p0, w.sigma, mode=1, leaf=4)[2]
    c16 = oracle.rhs(w.q0, w.p0, w.sigma, mode=1, leaf=16)[2]
    assert c1[1] >= c4[1] >= c16[1] and c1[0] <= c4[0] <= c16[0]


def _far_angle(x32, lo, hi, thr):
    s = np.float32(max(np.float32(hi[0] - lo[0]), np.float32(hi[1] - lo[1]),
                       np.float32(hi[2] - lo[2])))
    c = ((lo + hi).astype(np.float32) * np.float32(0.5)).astype(np.float32)
    d = (x32 - c).astype(np.float32)
    d2 = np.float32(d[0] * d[0])
    d2 = np.float32(d2 + np.float32(d[1] * d[1]))
    d2 = np.float32(d2 + np.float32(d[2] * d[2]))
    return bool(np.float32(s * s) < np.float32(thr * d2))


@pytest.mark.parametrize("theta", [0.3, 0.7])
def test_opening_angle_variant_lists(oracle, theta):
    """Opening-angle variant (classic Barnes-Hut form): sources partition the
    points; a summarised node passes the angle rule and none of its
    ancestors does; no node holding the target itself is summarised (a
    point inside a box has d <= sqrt(3)/2 s, so s^2 > theta^2 d^2 for theta <= 1)."""
    n = 300
    w = inputs.make("blobs", n, 31)
    q, p = w.q0, w.p0
    t = oracle.tree(q, p)
    t32 = np.float32(theta)
    thr = np.float32(t32 * t32)
    q32 = q.astype(np.float32)
    nfar = 0
    for m in range(0, n, 7):
        kind, ids = oracle.bh_list(q, p, w.sigma, m, theta, crit=1)
        seen = np.zeros(n, np.int64)
        for kd, i in zip(kind, ids):
            if kd == 1:
                nfar += 1
                assert _far_angle(q32[m], t["lo"][i], t["hi"][i], thr)
                members = t["order"][t["first"][i]:t["first"][i] + t["n"][i]]
                assert m not in members
                a = t["parent"][i]
                while a >= 0:
                    assert not _far_angle(q32[m], t["lo"][a], t["hi"][a], thr)
                    a = t["parent"][a]
                seen[members] += 1
            else:
                seen[i] += 1
        assert np.all(seen == 1)
    assert nfar > 0


def test_opening_angle_limits_and_error(oracle):
    w = inputs.make("blobs", 400, 37)
    Fe, Pe, _ = oracle.rhs(w.q0, w.p0, w.sigma)
    F0, P0, c0 = oracle.rhs(w.q0, w.p0, w.sigma, mode=1, thresh=1e-30, crit=1)
    assert c0[1] == 0 and c0[0] == 400 * 400
    np.testing.assert_allclose(F0, Fe, rtol=1e-12, atol=1e-15 * np.abs(Fe).max())
    errs = []
    for theta in (0.9, 0.5, 0.25):
        F, _, _ = oracle.rhs(w.q0, w.p0, w.sigma, mode=1, thresh=theta, crit=1)
        errs.append(np.abs(F - Fe).max())
    assert errs[0] > errs[1] > errs[2]


def _splitmix64(key):
    """splitmix64 (Steele, Lea and Flood, OOPSLA 2014): the generator's output
    for state `key`, in Python integers modulo 2**64."""
    m = (1 << 64) - 1
    z = (key + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


@pytest.mark.parametrize("geom,n,leaf,crit,thresh", [("blobs", 250, 1, 0, 3.0),
                                                     ("slab", 300, 1, 0, 2.0),
                                                     ("blobs", 220, 4, 0, 3.0),
                                                     ("ellipsoid", 200, 1, 1, 0.6)])
def test_decision_tally_matches_interaction_lists(oracle, geom, n, leaf, crit, thresh):
    """The per-target decision record (counts and fingerprints) equals the one
    recomputed here from each target's interaction list and the exported
    tree: a point's key is its DFS position, a node's its first DFS position
    and member count.  Duplicated points put a depth-10 list in the tree."""
    w = inputs.make(geom, n, 17)
    q = w.q0.copy()
    q[5] = q[2]
    q[6] = q[2]
    tally = oracle.bh_tally(q, w.sigma, thresh, leaf=leaf, crit=crit)
    t = oracle.tree(q, np.zeros_like(q))
    pos = np.empty(n, np.int64)
    pos[t["order"]] = np.arange(n)
    mask = (1 << 64) - 1
    for m in range(n):
        kind, ids = oracle.bh_list(q, w.p0, w.sigma, m, thresh, leaf=leaf, crit=crit)
        hp = hn = 0
        for k, i in zip(kind, ids):
            if k == 0:
                hp = (hp + _splitmix64((int(pos[i]) << 32) | 1)) & mask
            else:
                hn = (hn + _splitmix64((int(t["first"][i]) << 32) | int(t["n"][i]))) & mask
        want = [int((kind == 0).sum()), int((kind == 1).sum()), hp, hn]
        got = [int(tally[m, 0]), int(tally[m, 1]), int(tally[m, 2]) & mask,
               int(tally[m, 3]) & mask]  # (column 4: nodes reached, pinned below)
        assert got == want, m



@pytest.mark.parametrize("geom,n,leaf,thresh", [("blobs", 160, 1, 3.0), ("slab", 200, 1, 2.0),
                                                ("blobs", 150, 4, 3.0)])
def test_decision_tally_counts_by_independent_recursion(oracle, geom, n, leaf, thresh):
    """Points taken, nodes summarised and nodes reached per target, recounted
    by a recursion over the exported tree written here (FP32 far test in
    numpy float32, one rounding per operation): the traversal's node visits
    that the GPU walk's work is compared with."""
    w = inputs.make(geom, n, 23)
    q = w.q0.copy()
    q[5] = q[2]
    t = oracle.tree(q, np.zeros_like(q))
    M = len(t["n"])
    kids = [[] for _ in range(M)]
    for k in range(1, M):
        kids[int(t["parent"][k])].append(k)
    r = np.float32(thresh * w.sigma)
    thr = np.float32(r * r)
    q32 = q.astype(np.float32)

    def far(x, k):
        d = [max(np.float32(t["lo"][k][a] - x[a]), np.float32(0), np.float32(x[a] - t["hi"][k][a]))
             for a in range(3)]
        d2 = np.float32(np.float32(d[0] * d[0]) + np.float32(d[1] * d[1]))
        return np.float32(d2 + np.float32(d[2] * d[2])) > thr

    tally = oracle.bh_tally(q, w.sigma, thresh, leaf=leaf)
    for m in range(n):
        cnt = [0, 0, 0]  # points, nodes, reached

        def visit(k):
            nk = int(t["n"][k])
            if nk == 0:
                return
            # a chain of single-child cells (same members) counts once, at its top
            if nk >= 2 and (k == 0 or t["nchild"][int(t["parent"][k])] >= 2):
                cnt[2] += 1
            if nk >= 2 and far(q32[m], k):
                cnt[1] += 1
                return
            if t["leaf"][k] or nk <= leaf:
                cnt[0] += nk
                return
            for c in kids[k]:
                visit(c)
        visit(0)
        assert [int(tally[m, 0]), int(tally[m, 1]), int(tally[m, 4])] == cnt, m
