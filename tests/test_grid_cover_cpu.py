"""The cell rule of the truncation grid (option trunc_grid), restated in
numpy FP32: cells of side 0.51 r (doubled while there would be more than
8 N + 4096 of them), cell coordinates min(trunc((x - lo) * (1/h)), n - 1),
a stable sort by cell id and, for each block of 32 consecutive sorted
points, the rows of cells within two cells of theirs.  The swept pairs that
pass the FP32 truncation test are exactly the pairs a brute-force double
loop keeps, and every cell-range lookup stays inside the cell array.  (The
device kernels are checked against the oracle on the GPU.)"""
import numpy as np
import pytest

from paper_1907_04834_gb300 import inputs

f32 = np.float32


def _within(a, b, thr):
    d = (a - b).astype(f32)
    return (f32(d[..., 0] * d[..., 0]) + f32(d[..., 1] * d[..., 1])) + f32(d[..., 2] * d[..., 2]) \
        <= thr


def _grid_pairs(q, sigma, thresh=3.0):
    N = len(q)
    raw = q.astype(f32)
    r = f32(thresh * sigma)
    thr = f32(r * r)
    lo, hi = raw.min(0), raw.max(0)
    cap = min(8 * N + 4096, 1 << 30)
    inv = f32(f32(1.0) / f32(f32(0.51) * r))
    for _ in range(80):
        n = [min(max(float(f32(f32(hi[a] - lo[a]) * inv)), 0.0), 1e6) for a in range(3)]
        n = [int(u) + 1 for u in n]
        if n[0] * n[1] * n[2] <= cap:
            break
        inv = f32(inv * f32(0.5))
    else:
        n, inv = [1, 1, 1], f32(0)
    C = n[0] * n[1] * n[2]
    u = ((raw - lo).astype(f32) * inv).astype(f32)
    k = np.minimum(np.where(u >= 0, u, 0).astype(np.int64), np.array(n) - 1)
    key = (k[:, 2] * n[1] + k[:, 1]) * n[0] + k[:, 0]
    perm = np.argsort(key, kind="stable")
    ks = key[perm]
    cstart = np.searchsorted(ks, np.arange(C + 1), side="left")
    kept = 0
    for first in range(0, N, 32):
        kk = ks[first:first + 32]
        c = np.stack([kk % n[0], (kk // n[0]) % n[1], kk // (n[0] * n[1])], 1)
        lo_c = np.maximum(c.min(0) - 2, 0)
        hi_c = np.minimum(c.max(0) + 2, np.array(n) - 1)
        src = []
        for z in range(lo_c[2], hi_c[2] + 1):
            for y in range(lo_c[1], hi_c[1] + 1):
                row = (z * n[1] + y) * n[0]
                assert row + hi_c[0] + 1 <= C
                src.append(perm[cstart[row + lo_c[0]]:cstart[row + hi_c[0] + 1]])
        src = np.concatenate(src)
        assert len(np.unique(src)) == len(src)
        kept += int(_within(raw[perm[first:first + 32]][:, None], raw[src][None], thr).sum())
    brute = int(_within(raw[:, None], raw[None], thr).sum())
    return kept, brute, C


def _cases():
    rng = np.random.default_rng(0)
    out = [("N1", np.zeros((1, 3)), 1.0), ("N2", np.array([[0.0, 0, 0], [2.9, 0, 0]]), 1.0)]
    for geom, n, seed in [("slab", 777, 2), ("blobs", 1500, 5), ("ellipsoid", 600, 3)]:
        w = inputs.make(geom, n, seed)
        out.append((f"{geom}{n}", w.q0, w.sigma))
    flat = rng.normal(size=(400, 3)) * 3.0
    flat[:, 2] = 1.25
    out.append(("flat_z", flat, 1.0))
    out.append(("coincident", np.repeat(rng.normal(size=(5, 3)), 40, axis=0), 0.5))
    out.append(("sparse_cube", rng.uniform(-20.0, 20.0, size=(200, 3)), 1.0))
    out.append(("far_clusters", np.concatenate([rng.normal(size=(60, 3)) + 1e5 * k
                                                for k in range(3)]), 1.0))
    return [pytest.param(q, s, id=name) for name, q, s in out]


@pytest.mark.parametrize("q,sigma", _cases())
def test_grid_sweep_keeps_exactly_the_truncated_pairs(q, sigma):
    kept, brute, C = _grid_pairs(q, sigma)
    assert kept == brute
    assert 1 <= C <= 8 * len(q) + 4096
