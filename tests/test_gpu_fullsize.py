"""Full-size checks at the benchmark's N = 100,000 blob workload (sigma =
1.5, T = 20), in the configuration the benchmark times: sampled rows of one
exact right-hand side and one adjoint right-hand side against the oracle,
the Barnes-Hut right-hand sides at full size (interaction counts exact) and
a Barnes-Hut gradient over T = 4 steps against the oracle, and properties
of the full gradient that hold at any size.  Each test prints the measured
error beside its tolerance (pytest -s)."""
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
    eF = np.abs(F - Fo).max() / np.abs(Fo).max()
    eA = np.abs(npy(dA)[rows] - dAo).max() / np.abs(dAo).max()
    eB = np.abs(npy(dB)[rows] - dBo).max() / np.abs(dBo).max()
    print(f"\nexact RHS at N=100k, 200 rows: F {eF:.2e}, dA {eA:.2e}, dB {eB:.2e} (tol 1e-5)")
    assert eA <= 1e-5 and eB <= 1e-5


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


def test_bh_rhs_full_size(oracle, w):
    """Barnes-Hut forward and adjoint right-hand sides at N = 100,000 against
    the oracle's pointer-tree traversal: the same decisions (interaction
    counts equal) and values to FP32 rounding."""
    F, Phi, cnt = gs.rhs(dt(w.q0), dt(w.p0), w.sigma, mode="bh")
    Fo, Phio, cnto = oracle.rhs(w.q0, w.p0, w.sigma, mode=oracle.BH)
    assert tuple(cnt) == tuple(int(c) for c in cnto)
    eF = np.abs(npy(F) - Fo).max() / np.abs(Fo).max()
    eP = np.abs(npy(Phi) - Phio).max() / np.abs(Phio).max()
    rng = np.random.default_rng(1)
    al, be = rng.normal(size=w.q0.shape), rng.normal(scale=0.1, size=w.q0.shape)
    dA, dB, cnta = gs.adj_rhs(dt(w.q0), dt(w.p0), dt(al), dt(be), w.sigma, mode="bh")
    dAo, dBo, cntao = oracle.adj_rhs(w.q0, w.p0, al, be, w.sigma, mode=oracle.BH)
    assert tuple(cnta) == tuple(int(c) for c in cntao)
    eA = np.abs(npy(dA) - dAo).max() / np.abs(dAo).max()
    eB = np.abs(npy(dB) - dBo).max() / np.abs(dBo).max()
    print(f"\nBH RHS at N=100k: counts {tuple(cnt)}; F {eF:.2e}, Phi {eP:.2e}, dA {eA:.2e}, "
          f"dB {eB:.2e} (tol 1e-5)")
    assert max(eF, eP, eA, eB) <= 1e-5


def test_bh_gradient_full_size(oracle, w):
    """The whole Barnes-Hut shooting gradient at N = 100,000 (T = 4 steps to
    keep the oracle's time short) against the oracle."""
    T = 4
    E, g, q1 = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, T, w.lam, mode="bh")
    Eo, go, q1o = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, T, w.lam, mode=oracle.BH)
    dq = np.abs(npy(q1) - q1o).max() / w.sigma
    eg = np.linalg.norm(npy(g) - go) / np.linalg.norm(go)
    eE = abs(float(E[0]) - Eo[0]) / abs(Eo[0])
    print(f"\nBH gradient at N=100k, T={T}: max|dq1|/sigma {dq:.2e} (tol 1e-5), grad rel L2 "
          f"{eg:.2e} (tol 1e-4), E rel {eE:.2e}")
    assert dq <= 1e-5 and eg <= 1e-4 and eE <= 1e-6


def test_exact_gradient_slab20k(oracle):
    """The exact shooting gradient on the 20,000-point slab (sigma = 2; T = 4
    steps to keep the oracle's time short) against the FP64 oracle."""
    v = inputs.config("slab20k")
    T = 4
    E, g, q1 = gs.shoot_grad(dt(v.q0), dt(v.p0), dt(v.X), v.sigma, T, v.lam)
    Eo, go, q1o = oracle.shoot_grad(v.q0, v.p0, v.X, v.sigma, T, v.lam)
    dq = np.abs(npy(q1) - q1o).max() / v.sigma
    eg = np.linalg.norm(npy(g) - go) / np.linalg.norm(go)
    eE = abs(float(E[0]) - Eo[0]) / abs(Eo[0])
    print(f"\nexact gradient at N=20k, T={T}: max|dq1|/sigma {dq:.2e} (tol 1e-5), grad rel L2 "
          f"{eg:.2e} (tol 1e-4), E rel {eE:.2e}")
    assert dq <= 1e-5 and eg <= 1e-4 and eE <= 1e-6


def test_exact_rhs_sampled_rows_1m(oracle):
    """The exact forward and adjoint right-hand sides at the largest workload
    (sphere1m, N = 1,000,000: 10^12 pairs per launch), 200 sampled rows
    against the oracle's FP64 sums over all sources."""
    v = inputs.config("sphere1m")
    rng = np.random.default_rng(5)
    rows = np.sort(rng.choice(v.N, 200, replace=False))
    rows[-1] = v.N - 1
    F, Phi, _ = gs.rhs(dt(v.q0), dt(v.p0), v.sigma)
    Fo, Phio = oracle.rhs_rows(v.q0, v.p0, v.sigma, rows)
    eF = np.abs(npy(F)[rows] - Fo).max() / np.abs(Fo).max()
    eP = np.abs(npy(Phi)[rows] - Phio).max() / np.abs(Phio).max()
    al = rng.normal(size=v.q0.shape)
    be = rng.normal(scale=0.1, size=v.q0.shape)
    dA, dB, _ = gs.adj_rhs(dt(v.q0), dt(v.p0), dt(al), dt(be), v.sigma)
    dAo, dBo = oracle.adj_rhs_rows(v.q0, v.p0, al, be, v.sigma, rows)
    eA = np.abs(npy(dA)[rows] - dAo).max() / np.abs(dAo).max()
    eB = np.abs(npy(dB)[rows] - dBo).max() / np.abs(dBo).max()
    print(f"\nexact RHS at N=1M, 200 rows: F {eF:.2e}, Phi {eP:.2e}, dA {eA:.2e}, dB {eB:.2e} "
          f"(tol 1e-5)")
    assert max(eF, eP, eA, eB) <= 1e-5


def test_bh_rhs_1m(oracle):
    """The Barnes-Hut forward right-hand side at the largest workload
    (sphere1m, N = 1,000,000) against the oracle's pointer-tree traversal:
    the same decisions (interaction counts equal) and values to FP32
    rounding."""
    v = inputs.config("sphere1m")
    F, Phi, cnt = gs.rhs(dt(v.q0), dt(v.p0), v.sigma, mode="bh")
    Fo, Phio, cnto = oracle.rhs(v.q0, v.p0, v.sigma, mode=oracle.BH)
    assert tuple(cnt) == tuple(int(c) for c in cnto)
    eF = np.abs(npy(F) - Fo).max() / np.abs(Fo).max()
    eP = np.abs(npy(Phi) - Phio).max() / np.abs(Phio).max()
    print(f"\nBH RHS at N=1M: counts {tuple(cnt)}; F {eF:.2e}, Phi {eP:.2e} (tol 1e-5)")
    assert max(eF, eP) <= 1e-5
