"""Full-size checks at the benchmark's N = 100,000 blob workload (sigma =
1.5, T = 20), in the configuration the benchmark times: sampled rows of one
exact right-hand side and one adjoint right-hand side against the oracle,
and properties of the full gradient that hold at any size."""
import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt, npy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def w():
    return inputs.config("blobs100k")


def test_sampled_rows_rhs(oracle, w):
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(w.N, 200, replace=False))
    rows[-1] = w.N - 1
    F, Phi, _ = gs.rhs(dt(w.q0), dt(w.p0), w.sigma)
    Fo, Phio = oracle.rhs_rows(w.q0, w.p0, w.sigma, rows)
    F, Phi = npy(F)[rows], npy(Phi)[rows]
    assert np.abs(F - Fo).max() <= 1e-5 * np.abs(Fo).max()
    assert np.abs(Phi - Phio).max() <= 1e-5 * np.abs(Phio).max()
    al = rng.normal(size=w.q0.shape)
    be = rng.normal(scale=0.1, size=w.q0.shape)
    dA, dB, _ = gs.adj_rhs(dt(w.q0), dt(w.p0), dt(al), dt(be), w.sigma)
    dAo, dBo = oracle.adj_rhs_rows(w.q0, w.p0, al, be, w.sigma, rows)
    assert np.abs(npy(dA)[rows] - dAo).max() <= 1e-5 * np.abs(dAo).max()
    assert np.abs(npy(dB)[rows] - dBo).max() <= 1e-5 * np.abs(dBo).max()


def test_full_gradient_properties(w):
    """Deterministic (bit-identical reruns), checkpoint-exact, and the total
    momentum sum_i p_i is conserved by the forward flow."""
    args = (dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam)
    E1, g1, q1 = gs.shoot_grad(*args)
    E2, g2, q2 = gs.shoot_grad(*args)
    assert torch.equal(g1, g2) and torch.equal(E1, E2)
    E3, g3, _ = gs.shoot_grad(*args, ckpt_every=5)
    assert torch.equal(g1, g3)
    assert torch.isfinite(g1).all() and torch.isfinite(E1).all()
    _, p1, _ = gs.shoot(dt(w.q0), dt(w.p0), w.sigma, w.T)
    s0, s1 = w.p0.sum(axis=0), npy(p1).sum(axis=0)
    assert np.abs(s1 - s0).max() <= 1e-6 * np.abs(w.p0).sum()
