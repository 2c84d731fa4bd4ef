"""Semi-implicit symplectic Euler shooting (gs_params.sympl_iters, a variant of
the time discretisation of Sec. 2.1) against the oracle: trajectories and H
for the exact and Barnes-Hut right-hand sides, zero passes identical to the
explicit Euler path, the energy behaviour of the two schemes on a strongly
moving cloud, and the entry points that refuse the option."""
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
    """Only gs_shoot takes sympl_iters != 0; the gradient refuses it."""
    w = inputs.make("blobs", 300, 2)
    q, p, X = dt(w.q0), dt(w.p0), dt(w.X)
    c = gs_api.context(q.device.index)
    prm = make_params(w.sigma, 4, "exact", 1.0, sympl_iters=2)
    E = torch.zeros(3, dtype=torch.float64, device=q.device)
    g = torch.zeros_like(q)
    st = c.lib.gs_shoot_grad(c.handle, ctypes.c_void_p(q.data_ptr()),
                             ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                             q.shape[0], ctypes.byref(prm), ctypes.c_void_p(E.data_ptr()),
                             ctypes.c_void_p(g.data_ptr()), None, None)
    assert st == GS_ERR_UNSUPPORTED
    with pytest.raises(Exception):
        gs.shoot(q, p, w.sigma, 4, sympl_iters=65)
