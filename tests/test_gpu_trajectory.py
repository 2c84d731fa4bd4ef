"""Whole trajectories and gradients at the workloads' own lengths against the
oracle (Sec. 2.1 Eq. 1-2 with T Euler steps; Sec. 2.2 at every step in
Barnes-Hut mode), and the discrete path itself.

The Barnes-Hut forward map is discontinuous (a decision flips when a point
crosses a node's threshold), so a long trajectory is where the CUDA path and
the oracle could part: the tests here run the benchmark's blobs100k at its
T = 20, the 20k slab at its T = 20, the 1M sphere's gradient through the
checkpointed adjoint, and a blob cloud whose momenta move the points by
about a kernel width, comparing decisions target by target at every step.
Each prints its measured errors beside the tolerances (pytest -s)."""
import time

import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt, npy

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,M", [("exact", 0), ("bh", 0), ("bh", 2)])
def test_traj_ends_where_shoot_ends(mode, M):
    w = inputs.make("blobs", 3000, 21, T=12)
    qt, pt = gs.shoot_traj(dt(w.q0), dt(w.p0), w.sigma, w.T, mode=mode, sympl_iters=M)
    q1, p1, _ = gs.shoot(dt(w.q0), dt(w.p0), w.sigma, w.T, mode=mode, sympl_iters=M)
    assert qt.shape == (w.T + 1, w.N, 3)
    assert torch.equal(qt[0], dt(w.q0)) and torch.equal(pt[0], dt(w.p0))
    assert torch.equal(qt[-1], q1) and torch.equal(pt[-1], p1)


def test_traj_intermediate_states(oracle):
    """State k of the path equals the oracle's Euler path after k steps."""
    w = inputs.make("slab", 1500, 22, T=8)
    qt, pt = gs.shoot_traj(dt(w.q0), dt(w.p0), w.sigma, w.T, mode="bh")
    qt, pt = npy(qt), npy(pt)
    q, p = w.q0.copy(), w.p0.copy()
    h = 1.0 / w.T
    for k in range(w.T + 1):
        assert np.abs(qt[k] - q).max() <= 1e-5 * w.sigma, k
        F, Phi, _ = oracle.rhs(q, p, w.sigma, mode=oracle.BH)
        q, p = q + h * F, p + h * Phi


def _grad_check(oracle, w, mode, T, ckpt=0):
    t0 = time.time()
    E, g, q1 = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, T, w.lam, mode=mode,
                             ckpt_every=ckpt)
    E, g, q1 = npy(E), npy(g), npy(q1)
    t1 = time.time()
    Eo, go, q1o = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, T, w.lam,
                                    mode=oracle.BH if mode == "bh" else oracle.EXACT)
    t2 = time.time()
    dq = np.abs(q1 - q1o).max() / w.sigma
    eg = np.linalg.norm(g - go) / np.linalg.norm(go)
    eE = abs(E[0] - Eo[0]) / abs(Eo[0])
    print(f"\n{w.name} {mode} gradient, T={T}, ckpt_every={ckpt}: max|dq1|/sigma {dq:.2e} "
          f"(tol 1e-5), grad rel L2 {eg:.2e} (tol 1e-4), E rel {eE:.2e}; "
          f"GPU {t1 - t0:.1f} s, oracle {t2 - t1:.1f} s on {oracle.num_threads()} threads")
    assert dq <= 1e-5 and eg <= 1e-4 and eE <= 1e-6


def test_bh_gradient_blobs100k_full_length(oracle):
    """The benchmark's own gradient: blobs100k, Barnes-Hut, T = 20."""
    w = inputs.config("blobs100k")
    _grad_check(oracle, w, "bh", w.T)


def test_exact_gradient_slab20k_full_length(oracle):
    """The 20k slab's exact gradient at its stated T = 20."""
    w = inputs.config("slab20k")
    _grad_check(oracle, w, "exact", w.T)


def test_bh_gradient_sphere1m_checkpointed(oracle):
    """The 1M-point sphere's Barnes-Hut gradient through the checkpointed
    adjoint (every 3rd state kept, the others recomputed), T = 6 so the
    oracle ends in minutes."""
    w = inputs.config("sphere1m")
    _grad_check(oracle, w, "bh", 6, ckpt=3)


def test_deforming_blobs_decisions_along_trajectory(oracle):
    """Blobs (N = 100,000) with momenta 20x the benchmark's, so the points
    move by about a kernel width over t in [0, 1] (T = 20; median 0.8
    sigma, 90th percentile 1.9 sigma in the oracle): at every state of
    the CUDA path its decisions equal the oracle's on that same state,
    target by target; against the oracle's own path (states that differ by
    rounding) the number of targets whose decisions differ is reported, and
    the end points agree within 1e-5 sigma."""
    w = inputs.config("blobs100k")
    p0 = 20.0 * w.p0
    qt, _ = gs.shoot_traj(dt(w.q0), dt(p0), w.sigma, w.T, mode="bh")
    qt = npy(qt)
    q, p = w.q0.copy(), p0.copy()
    h = 1.0 / w.T
    moved = np.linalg.norm(qt[-1] - w.q0, axis=1) / w.sigma
    flips = []
    for k in range(w.T + 1):
        tg = npy(gs.bh_tally(dt(qt[k]), w.sigma))
        to_same = oracle.bh_tally(qt[k], w.sigma)
        bad = int(np.any(tg != to_same, axis=1).sum())
        assert bad == 0, (k, bad)
        to_own = oracle.bh_tally(q, w.sigma)
        flips.append(int(np.any(tg != to_own, axis=1).sum()))
        if k < w.T:
            F, Phi, _ = oracle.rhs(q, p, w.sigma, mode=oracle.BH)
            q, p = q + h * F, p + h * Phi
    dq = np.abs(qt[-1] - q).max() / w.sigma
    print(f"\ndeforming blobs100k (20x momenta): displacement median {np.median(moved):.2f} "
          f"sigma, max {moved.max():.2f} sigma; targets whose decisions differ between the "
          f"CUDA and oracle paths per step: {flips}; max|dq1|/sigma {dq:.2e} (tol 1e-5)")
    assert dq <= 1e-5
