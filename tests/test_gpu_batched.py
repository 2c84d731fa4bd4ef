"""Many independent registrations in one call (gs_shoot_batched): every
subject's objective and gradient against the FP64 oracle run on that subject
alone (points interact only within their subject), through the C ABI.

The exact path runs one persistent launch per step over (subject, target
tile) work items; the Barnes-Hut path builds one forest of all subjects per
step, in which every subject's tree, decisions and sums are those it would
have alone (checked bit for bit against single-set calls).
Tolerances as for one point set: gradient relative L2 <= 1e-4, E to 1e-6."""
import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt, npy, rel_l2

pytestmark = pytest.mark.gpu


def _stack(ws):
    off = np.zeros(len(ws) + 1, np.int64)
    off[1:] = np.cumsum([w.N for w in ws])
    cat = lambda k: np.concatenate([getattr(w, k) for w in ws])
    return cat("q0"), cat("p0"), cat("X"), off


def _subjects(T=6):
    # ragged sizes: one point, two, a tile and one, a tile of targets short,
    # several tiles with a tail; different geometries and centres
    specs = [("slab", 1, 31), ("slab", 2049, 32), ("blobs", 700, 33), ("slab", 2, 34),
             ("ellipsoid", 513, 35), ("slab", 1500, 36), ("blobs", 255, 37)]
    ws = []
    for k, (g, n, seed) in enumerate(specs):
        w = inputs.make(g, n, seed, T=T, sigma=2.0)
        w.q0 = w.q0 + 100.0 * k  # subjects far apart would not interact anyway
        w.X = w.X + 100.0 * k
        ws.append(w)
    return ws


@pytest.mark.parametrize("mode", ["exact", "bh"])
def test_batched_matches_oracle_per_subject(oracle, mode):
    ws = _subjects()
    q0, p0, X, off = _stack(ws)
    T, sigma, lam = ws[0].T, 2.0, ws[0].lam
    E, g = gs.shoot_batched(dt(q0), dt(p0), dt(X), off, sigma, T, lam, mode=mode)
    E, g = npy(E), npy(g)
    for k, w in enumerate(ws):
        if mode == "exact":
            Eo, go, _ = oracle.shoot_grad(w.q0, w.p0, w.X, sigma, T, lam)
        else:
            Eo, go, _ = oracle.shoot_grad(w.q0, w.p0, w.X, sigma, T, lam, mode=oracle.BH)
        gk = g[off[k]:off[k + 1]]
        assert rel_l2(gk, go) <= 1e-4, (k, w.N)
        np.testing.assert_allclose(E[k], Eo, rtol=1e-6, err_msg=f"subject {k}")


def test_batched_subjects_do_not_interact(oracle):
    """Two identical subjects placed on top of each other give the result of
    one subject alone, twice."""
    w = inputs.make("slab", 900, 41, T=5)
    q0, p0, X, off = _stack([w, w])
    E, g = gs.shoot_batched(dt(q0), dt(p0), dt(X), off, w.sigma, w.T, w.lam)
    E, g = npy(E), npy(g)
    assert np.array_equal(E[0], E[1])
    assert np.array_equal(g[:900], g[900:])
    Eo, go, _ = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, w.lam)
    assert rel_l2(g[:900], go) <= 1e-4
    np.testing.assert_allclose(E[0], Eo, rtol=1e-6)


def test_batched_is_deterministic_and_checkpointing_bit_exact():
    """The work queue hands items to blocks in a run-dependent order, but
    each item's sums are fixed: repeated calls, and checkpointed calls, are
    bit-identical."""
    ws = _subjects(T=7)
    q0, p0, X, off = _stack(ws)
    args = (dt(q0), dt(p0), dt(X), off, 2.0, 7, ws[0].lam)
    E0, g0 = gs.shoot_batched(*args)
    E1, g1 = gs.shoot_batched(*args)
    assert torch.equal(E0, E1) and torch.equal(g0, g1)
    for ck in (1, 3):
        E2, g2 = gs.shoot_batched(*args, ckpt_every=ck)
        assert torch.equal(E0, E2) and torch.equal(g0, g2), ck


def test_batched_bh_equals_single_subject_calls():
    ws = _subjects(T=4)
    q0, p0, X, off = _stack(ws)
    E, g = gs.shoot_batched(dt(q0), dt(p0), dt(X), off, 2.0, 4, ws[0].lam, mode="bh")
    for k, w in enumerate(ws):
        Ek, gk, _ = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), 2.0, 4, w.lam, mode="bh")
        assert torch.equal(E[k], Ek) and torch.equal(g[off[k]:off[k + 1]], gk), k


def test_batched_bh_forest_overlapping_subjects():
    """Subjects that overlap in space (same region, different clouds) still
    interact only within themselves: forest result == single-set calls."""
    ws = [inputs.make("blobs", n, 50 + n, T=3) for n in (1200, 900, 1)]
    q0, p0, X, off = _stack(ws)
    E, g = gs.shoot_batched(dt(q0), dt(p0), dt(X), off, ws[0].sigma, 3, 1.0, mode="bh")
    for k, w in enumerate(ws):
        Ek, gk, _ = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, 3, 1.0, mode="bh")
        assert torch.equal(E[k], Ek) and torch.equal(g[off[k]:off[k + 1]], gk), k


@pytest.mark.parametrize("mode", ["exact", "bh"])
def test_batched_many_small_subjects(oracle, mode):
    """300 subjects of 1-60 points (the forest's sort takes two subject
    passes), against the oracle subject by subject."""
    rng = np.random.default_rng(77)
    ws = [inputs.make("slab", int(n), 1000 + k, T=2, sigma=2.0)
          for k, n in enumerate(rng.integers(1, 61, size=300))]
    q0, p0, X, off = _stack(ws)
    E, g = gs.shoot_batched(dt(q0), dt(p0), dt(X), off, 2.0, 2, 1.0, mode=mode)
    E, g = npy(E), npy(g)
    om = oracle.BH if mode == "bh" else oracle.EXACT
    for k, w in enumerate(ws):
        Eo, go, _ = oracle.shoot_grad(w.q0, w.p0, w.X, 2.0, 2, 1.0, mode=om)
        assert rel_l2(g[off[k]:off[k + 1]], go) <= 1e-4, k
        np.testing.assert_allclose(E[k], Eo, rtol=1e-6, err_msg=f"subject {k}")


def test_batched_exact_close_to_single_subject_calls():
    """The batched kernel sums each subject's sources in one pass, the
    single-set kernel in split partials: equal up to FP32 rounding."""
    ws = _subjects(T=5)
    q0, p0, X, off = _stack(ws)
    E, g = gs.shoot_batched(dt(q0), dt(p0), dt(X), off, 2.0, 5, ws[0].lam)
    for k, w in enumerate(ws):
        Ek, gk, _ = gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), 2.0, 5, w.lam)
        assert rel_l2(npy(g[off[k]:off[k + 1]]), npy(gk)) <= 2e-6, k
        np.testing.assert_allclose(npy(E[k]), npy(Ek), rtol=1e-9)


def test_batched_host_buffers_match_device_buffers():
    ws = _subjects(T=3)[:4]
    q0, p0, X, off = _stack(ws)
    Ed, gd = gs.shoot_batched(dt(q0), dt(p0), dt(X), off, 2.0, 3)
    c = lambda a: torch.as_tensor(a, dtype=torch.float64)
    Eh, gh = gs.shoot_batched(c(q0), c(p0), c(X), off, 2.0, 3)
    assert not gh.is_cuda
    assert torch.equal(Eh, Ed.cpu()) and torch.equal(gh, gd.cpu())


def test_batched_invalid_offsets_raise():
    w = inputs.make("slab", 10, 1)
    q, p, X = dt(w.q0), dt(w.p0), dt(w.X)
    with pytest.raises(gs.GSError):
        gs.shoot_batched(q, p, X, [0, 5, 5, 10], w.sigma, 3)   # empty subject
    with pytest.raises(gs.GSError):
        gs.shoot_batched(q, p, X, [0, 7, 4, 10], w.sigma, 3)   # decreasing
    with pytest.raises(ValueError):
        gs.shoot_batched(q, p, X, [0, 5, 9], w.sigma, 3)       # does not end at N
    with pytest.raises(gs.GSError):
        gs.shoot_batched(q, p, X, [1, 5, 10], w.sigma, 3)      # does not start at 0
