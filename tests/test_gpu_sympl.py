"""Semi-implicit symplectic Euler shooting (gs_params.sympl_iters, a variant of
the time discretisation of Sec. 2.1) against the oracle: trajectories and H
for the exact and Barnes-Hut right-hand sides, zero passes identical to the
explicit Euler path, the energy behaviour of the two schemes on a strongly
moving cloud, the gradient through the scheme (discrete adjoint of its
passes) against the oracle's, and the entry points that refuse the option."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import api as gs_api, inputs
from paper_1907_04834_gb300._lib import make_params, GS_ERR_UNSUPPORTED
from gpu_util import dt, npy

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["exact", "bh"])
def test_zero_passes_is_explicit_euler(mode):
    w = inputs.make("blobs", 1200, 21)
    a = gs.shoot(dt(w.q0), dt(w.p0), w.sigma, 6, mode=mode, with_H=True)
    b = gs.shoot(dt(w.q0), dt(w.p0), w.sigma, 6, mode=mode, with_H=True, sympl_iters=0)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("mode,geom,n,seed,M,leaf", [("exact", "blobs", 1500, 3, 2, 1),
                                                     ("exact", "slab", 2000, 4, 3, 1),
                                                     ("bh", "blobs", 3000, 7, 2, 1),
                                                     ("bh", "sphere", 3000, 6, 1, 1),
                                                     ("bh", "blobs", 2500, 8, 2, 8),
                                                     ("trunc", "blobs", 2000, 9, 2, 1)])
def test_sympl_matches_oracle(oracle, mode, geom, n, seed, M, leaf):
    w = inputs.make(geom, n, seed)
    T = 8
    q1, p1, H = gs.shoot(dt(w.q0), dt(w.p0), w.sigma, T, mode=mode, with_H=True, sympl_iters=M,
                         leaf_size=leaf)
    omode = {"exact": oracle.EXACT, "bh": oracle.BH, "trunc": oracle.TRUNC}[mode]
    q1o, p1o, Ho = oracle.shoot_sympl(w.q0, w.p0, w.sigma, T, M, mode=omode, leaf=leaf)
    dq = np.abs(npy(q1) - q1o).max() / w.sigma
    dp = np.abs(npy(p1) - p1o).max() / np.abs(p1o).max()
    eH = np.abs(npy(H) - Ho).max() / abs(Ho[0])
    print(f"\nsymplectic M={M} {mode} {geom}: max|dq|/sigma {dq:.2e}, p {dp:.2e}, H {eH:.2e}")
    assert dq <= 1e-5 and dp <= 1e-4 and eH <= 1e-5


def test_sympl_energy_on_strong_motion(oracle):
    """A small cloud with large momenta (strong deformation within t in
    [0, 1]): explicit Euler loses most of H, two fixed-point passes keep it to
    a fraction of a percent; the GPU's H values follow the oracle's."""
    rng = np.random.default_rng(1)
    q = rng.normal(scale=2.0, size=(40, 3))
    p = rng.normal(scale=3.0, size=(40, 3))
    rel = {}
    for M in (0, 2):
        _, _, H = gs.shoot(dt(q), dt(p), 1.0, 50, with_H=True, sympl_iters=M)
        _, _, Ho = oracle.shoot_sympl(q, p, 1.0, 50, M)
        H = npy(H)
        rel[M] = abs(H[1] - H[0]) / H[0]
        assert abs(H[1] - Ho[1]) <= 1e-3 * abs(Ho[0])
    print(f"\nrelative H drift over t in [0, 1]: explicit {rel[0]:.2e}, symplectic (2 passes) "
          f"{rel[2]:.2e}")
    assert rel[0] > 0.1 and rel[2] < 0.01


def test_sympl_refused_elsewhere():
    """The batched gradient refuses sympl_iters != 0 (gs_shoot, gs_shoot_traj
    and gs_shoot_grad take it), and an out-of-range count is an error."""
    w = inputs.make("blobs", 300, 2)
    q, p, X = dt(w.q0), dt(w.p0), dt(w.X)
    c = gs_api.context(q.device.index)
    prm = make_params(w.sigma, 4, "exact", 1.0, sympl_iters=2)
    E = torch.zeros((2, 3), dtype=torch.float64, device=q.device)
    g = torch.zeros_like(q)
    off = torch.tensor([0, 150, 300], dtype=torch.int64)
    st = c.lib.gs_shoot_batched(c.handle, 2, ctypes.c_void_p(off.data_ptr()),
                                ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                                ctypes.c_void_p(X.data_ptr()), ctypes.byref(prm),
                                ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                None)
    assert st == GS_ERR_UNSUPPORTED
    with pytest.raises(Exception):
        gs.shoot(q, p, w.sigma, 4, sympl_iters=65)


@pytest.mark.parametrize("mode,geom,n,seed,M,T,scale", [("exact", "blobs", 1500, 3, 2, 8, 1.0),
                                                        ("exact", "slab", 2000, 4, 3, 6, 5.0),
                                                        ("bh", "blobs", 3000, 7, 2, 8, 20.0),
                                                        ("bh", "sphere", 3000, 6, 1, 6, 1.0)])
def test_sympl_gradient_matches_oracle(oracle, mode, geom, n, seed, M, T, scale):
    """The objective's gradient through the semi-implicit scheme (discrete
    adjoint of the fixed-point passes) against the oracle's; scale
    multiplies the momenta so that the passes change the step."""
    w = inputs.make(geom, n, seed)
    p0 = scale * w.p0
    E, g, q1 = gs.shoot_grad(dt(w.q0), dt(p0), dt(w.X), w.sigma, T, w.lam, mode=mode,
                             sympl_iters=M)
    omode = oracle.EXACT if mode == "exact" else oracle.BH
    Eo, go, q1o = oracle.shoot_grad_sympl(w.q0, p0, w.X, w.sigma, T, w.lam, M, mode=omode)
    _, ge, _ = oracle.shoot_grad(w.q0, p0, w.X, w.sigma, T, w.lam, mode=omode)
    dq = np.abs(npy(q1) - q1o).max() / w.sigma
    eg = np.linalg.norm(npy(g) - go) / np.linalg.norm(go)
    eE = abs(float(E[0]) - Eo[0]) / abs(Eo[0])
    dpass = np.linalg.norm(go - ge) / np.linalg.norm(go)
    print(f"\nsymplectic gradient M={M} {mode} {geom} N={n} T={T}: max|dq1|/sigma {dq:.2e}, "
          f"grad rel L2 {eg:.2e} (tol 1e-4), E rel {eE:.2e}; the passes move the gradient by "
          f"{dpass:.2e}")
    assert dq <= 1e-5 and eg <= 1e-4 and eE <= 1e-6


@pytest.mark.parametrize("mode", ["exact", "bh"])
def test_sympl_gradient_checkpointed_is_stored(mode):
    w = inputs.make("blobs", 2000, 12)
    args = (dt(w.q0), dt(20.0 * w.p0), dt(w.X), w.sigma, 7, w.lam)
    E1, g1, q1 = gs.shoot_grad(*args, mode=mode, sympl_iters=2)
    E2, g2, q2 = gs.shoot_grad(*args, mode=mode, sympl_iters=2, ckpt_every=3)
    assert torch.equal(g1, g2) and torch.equal(E1, E2) and torch.equal(q1, q2)
