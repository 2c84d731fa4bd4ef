"""Pins for the oracle's pure 3-sigma truncation (mode 2: only pairs whose
FP32 positions lie within the threshold), a variant compared against the
paper's Barnes-Hut approximation: pair counts by an independent float32
count, the exact limit, conservation of total momentum, an error bound
against the exact sums, and the adjoint against finite differences."""
import numpy as np
import pytest

from paper_1907_04834_gb300 import inputs
from test_oracle_flow import _rand_cloud


def _count_within(q, sigma, thresh):
    """Pairs (i, j), i = j included, with (dx^2 + dy^2) + dz^2 <= r^2 in float32."""
    q32 = q.astype(np.float32)
    r = np.float32(thresh * sigma)
    thr = np.float32(r * r)
    d = (q32[:, None, :] - q32[None, :, :]).astype(np.float32)
    sq = (d * d).astype(np.float32)
    d2 = ((sq[..., 0] + sq[..., 1]).astype(np.float32) + sq[..., 2]).astype(np.float32)
    return int(np.count_nonzero(d2 <= thr))


@pytest.mark.parametrize("geom,n,thresh", [("blobs", 400, 3.0), ("slab", 500, 2.0),
                                           ("ellipsoid", 300, 1.0)])
def test_pair_counts_and_momentum(oracle, geom, n, thresh):
    w = inputs.make(geom, n, 7)
    F, Phi, cnt = oracle.rhs(w.q0, w.p0, w.sigma, mode=oracle.TRUNC, thresh=thresh)
    assert cnt[0] == _count_within(w.q0, w.sigma, thresh) and cnt[1] == 0
    assert n <= cnt[0] < n * n  # every point with itself, not every pair
    # the relation is symmetric, Phi pairwise antisymmetric: sum Phi = 0
    assert np.abs(Phi.sum(0)).max() <= 1e-12 * np.abs(Phi).sum()
    rng = np.random.default_rng(1)
    al, be = rng.normal(size=w.q0.shape), rng.normal(size=w.q0.shape)
    _, _, cnta = oracle.adj_rhs(w.q0, w.p0, al, be, w.sigma, mode=oracle.TRUNC, thresh=thresh)
    assert cnta[0] == cnt[0]


def test_huge_threshold_is_exact_and_error_bound(oracle):
    w = inputs.make("blobs", 500, 8)
    Fe, Pe, _ = oracle.rhs(w.q0, w.p0, w.sigma)
    Fb, Pb, cb = oracle.rhs(w.q0, w.p0, w.sigma, mode=oracle.TRUNC, thresh=1e6)
    assert cb[0] == 500 * 500
    np.testing.assert_allclose(Fb, Fe, rtol=1e-13, atol=1e-15 * np.abs(Fe).max())
    np.testing.assert_allclose(Pb, Pe, rtol=1e-13, atol=1e-14 * np.abs(Pe).max())
    # a dropped pair is beyond r, where G < exp(-thresh^2 / 2)
    for thresh in (2.0, 3.0):
        Ft, _, _ = oracle.rhs(w.q0, w.p0, w.sigma, mode=oracle.TRUNC, thresh=thresh)
        bound = np.exp(-thresh ** 2 / 2) * np.abs(w.p0).sum(0) * (1 + 1e-6)
        assert np.all(np.abs(Ft - Fe) <= bound[None, :])


def test_far_clusters_move_independently(oracle):
    q, p = _rand_cloud(30, 3, scale=1.0)
    q2 = q + np.array([20.0, 0.0, 0.0])
    both = oracle.shoot(np.vstack([q, q2]), np.vstack([p, p]), 1.0, 6, mode=oracle.TRUNC)
    one = oracle.shoot(q, p, 1.0, 6, mode=oracle.TRUNC)
    assert np.array_equal(both[0][:30], one[0])


def test_truncated_gradient_matches_finite_differences(oracle):
    """Away from pairs crossing the cutoff the truncated objective is smooth,
    and its discrete adjoint is its exact gradient."""
    rng = np.random.default_rng(5)
    n, sigma, T, lam, th = 25, 1.0, 4, 1.0, 2.0
    q0 = rng.normal(scale=1.5, size=(n, 3))
    p0 = rng.normal(scale=0.2, size=(n, 3))
    X = q0 + rng.normal(scale=0.3, size=(n, 3))
    E, g, _ = oracle.shoot_grad(q0, p0, X, sigma, T, lam, mode=oracle.TRUNC, thresh=th)
    eps = 1e-6
    for k in range(8):
        v = rng.normal(size=(n, 3))
        v /= np.linalg.norm(v)
        Ep = oracle.shoot_grad(q0, p0 + eps * v, X, sigma, T, lam, mode=oracle.TRUNC, thresh=th)[0]
        Em = oracle.shoot_grad(q0, p0 - eps * v, X, sigma, T, lam, mode=oracle.TRUNC, thresh=th)[0]
        fd = (Ep[0] - Em[0]) / (2 * eps)
        assert fd == pytest.approx(float(np.sum(g * v)), rel=1e-6, abs=1e-9)
