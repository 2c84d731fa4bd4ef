"""Tile shape of the exact kernels and checkpoint spacing.

The number of source splits J of the exact forward and adjoint kernels
(options exact_splits_fwd / exact_splits_adj, chosen by gs_autotune_exact)
only regroups the FP32 tile partials: every J matches the oracle within the
stated tolerances and reruns are bit-identical.  ckpt_every = -1 keeps every
round(sqrt(T))-th state, and the recomputed trajectory gives the
store-everything gradient bit for bit."""
import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt, npy, max_rel, rel_l2, phi_floor

pytestmark = pytest.mark.gpu


def _with_splits(jf, ja, fn):
    gs.set_option("exact_splits_fwd", jf)
    gs.set_option("exact_splits_adj", ja)
    try:
        return fn()
    finally:
        gs.set_option("exact_splits_fwd", 0)
        gs.set_option("exact_splits_adj", 0)


# slab 3000: ceil(3000 / 512) = 6 source tiles, so J = 64 acts as 6
@pytest.mark.parametrize("jf,ja", [(1, 1), (2, 5), (6, 3), (64, 64)])
def test_splits_match_oracle(oracle, jf, ja):
    w = inputs.make("slab", 3000, 9, T=4)
    rng = np.random.default_rng(3)
    al, be = rng.normal(size=w.q0.shape), rng.normal(scale=0.1, size=w.q0.shape)

    def run():
        F, Phi, _ = gs.rhs(dt(w.q0), dt(w.p0), w.sigma)
        dA, dB, _ = gs.adj_rhs(dt(w.q0), dt(w.p0), dt(al), dt(be), w.sigma)
        E, g, q1 = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam)
        return F, Phi, dA, dB, E, g, q1

    F, Phi, dA, dB, E, g, q1 = _with_splits(jf, ja, run)
    again = _with_splits(jf, ja, run)
    for a, b in zip((F, Phi, dA, dB, E, g, q1), again):
        assert torch.equal(a, b)
    Fo, Phio, _ = oracle.rhs(w.q0, w.p0, w.sigma)
    dAo, dBo, _ = oracle.adj_rhs(w.q0, w.p0, al, be, w.sigma)
    Eo, go, q1o = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, w.lam)
    assert max_rel(npy(F), Fo) <= 1e-5
    assert max_rel(npy(Phi), Phio, phi_floor(w.p0, w.sigma)) <= 1e-5
    assert max_rel(npy(dA), dAo, 1e-12 * np.abs(al).max() * np.abs(w.p0).max() / w.sigma) <= 1e-5
    assert max_rel(npy(dB), dBo) <= 1e-5
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma
    assert rel_l2(npy(g), go) <= 1e-4
    assert abs(float(E[0]) - Eo[0]) <= 1e-6 * abs(Eo[0])


def test_autotune_exact_returns_applied_candidates():
    w = inputs.make("slab", 3000, 9, T=4)
    q, p, X = dt(w.q0), dt(w.p0), dt(w.X)
    before = gs.shoot_grad(q, p, X, w.sigma, w.T, w.lam)
    (jf, ja), ms = gs.autotune_exact(q, p, w.sigma, candidates=(1, 2, 4, 64))
    assert jf in (1, 2, 4, 6) and ja in (1, 2, 4, 6)  # 64 acts as the 6 source tiles
    assert all(t[0] > 0 and t[1] > 0 for t in ms.values())
    # the tuner restores the options: the default choice is unchanged
    after = gs.shoot_grad(q, p, X, w.sigma, w.T, w.lam)
    for a, b in zip(before, after):
        assert torch.equal(a, b)
    tuned = _with_splits(jf, ja, lambda: gs.shoot_grad(q, p, X, w.sigma, w.T, w.lam))
    assert rel_l2(npy(tuned[1]), npy(before[1])) <= 1e-5


def test_split_options_and_tuner_checked():
    for name in ("exact_splits_fwd", "exact_splits_adj"):
        for bad in (-1, 4097):
            with pytest.raises(gs.GSError):
                gs.set_option(name, bad)
    w = inputs.make("slab", 300, 2)
    with pytest.raises(gs.GSError):
        gs.autotune_exact(dt(w.q0), dt(w.p0), w.sigma, candidates=(0,))
    with pytest.raises(gs.GSError):
        gs.autotune_exact(dt(w.q0), dt(w.p0), w.sigma, candidates=tuple(range(1, 66)))


@pytest.mark.parametrize("mode,T", [("exact", 11), ("exact", 2), ("bh", 9)])
def test_ckpt_sqrt_T_is_bit_exact(mode, T):
    """ckpt_every = -1 (every round(sqrt(T))-th state: 3 for T = 9 and 11,
    1 for T = 2) equals the store-everything gradient bit for bit."""
    w = inputs.make("blobs", 1500, 23, T=T)
    args = (dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam)
    a = gs.shoot_grad(*args, mode=mode)
    b = gs.shoot_grad(*args, mode=mode, ckpt_every=-1)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    with pytest.raises(gs.GSError):
        gs.shoot_grad(*args, mode=mode, ckpt_every=-2)
