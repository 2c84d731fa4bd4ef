"""CUDA-graph replay of the step loops and the batched gradient-descent
driver, through the C ABI.

With graphs on (the default) an entry point captures its whole step loop
the first time it sees a set of sizes, parameters and device addresses and
replays the graph afterwards; results must be bit-identical to launching
kernel by kernel, also when the replayed inputs hold new values."""
import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from gpu_util import dt, npy

pytestmark = pytest.mark.gpu


def _eager(fn):
    gs.set_option("graphs", 0)
    try:
        return fn()
    finally:
        gs.set_option("graphs", 1)


def _same(a, b):
    return all(torch.equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("mode", ["exact", "bh"])
def test_shoot_and_grad_replay_bit_exact(mode):
    w = inputs.make("blobs", 1500, 61, T=6)
    q0, p0, X = dt(w.q0), dt(w.p0), dt(w.X)
    shoot = lambda: gs.shoot(q0, p0, w.sigma, w.T, mode=mode, with_H=True)
    grad = lambda: gs.shoot_grad(q0, p0, X, w.sigma, w.T, w.lam, mode=mode)
    grad_ck = lambda: gs.shoot_grad(q0, p0, X, w.sigma, w.T, w.lam, mode=mode, ckpt_every=4)
    for fn in (shoot, grad, grad_ck):
        ref = _eager(fn)
        first, again = fn(), fn()  # capture, then replay
        assert _same(ref, first) and _same(ref, again)
    # new values in the same buffers: the replay reads them
    p0.mul_(1.5)
    X.add_(0.25)
    for fn in (shoot, grad):
        ref = _eager(fn)
        assert _same(ref, fn())


@pytest.mark.parametrize("mode", ["exact", "bh"])
def test_batched_replay_bit_exact(mode):
    ws = [inputs.make("slab", n, 70 + n, T=4, sigma=2.0) for n in (700, 1, 1300)]
    off = np.zeros(4, np.int64)
    off[1:] = np.cumsum([w.N for w in ws])
    cat = lambda k: dt(np.concatenate([getattr(w, k) for w in ws]))
    q0, p0, X = cat("q0"), cat("p0"), cat("X")
    fn = lambda: gs.shoot_batched(q0, p0, X, off, 2.0, 4, 1.0, mode=mode)
    ref = _eager(fn)
    assert _same(ref, fn()) and _same(ref, fn())
    p0.mul_(-1.0)
    assert _same(_eager(fn), fn())
    # another layout: captured again
    off2 = np.array([0, 700, int(off[-1])], np.int64)
    fn2 = lambda: gs.shoot_batched(q0, p0, X, off2, 2.0, 4, 1.0, mode=mode)
    assert _same(_eager(fn2), fn2())


def test_host_buffers_with_graphs():
    w = inputs.make("slab", 600, 81, T=3)
    c = lambda a: torch.as_tensor(a, dtype=torch.float64)
    Eh, gh, qh = gs.shoot_grad(c(w.q0), c(w.p0), c(w.X), w.sigma, w.T, w.lam)
    Ed, gd, qd = _eager(lambda: gs.shoot_grad(dt(w.q0), dt(w.p0), dt(w.X), w.sigma, w.T, w.lam))
    assert torch.equal(gh, gd.cpu()) and torch.equal(Eh, Ed.cpu())


@pytest.mark.parametrize("mode", ["exact", "bh"])
def test_descend_matches_manual_loop(mode):
    """The native descent driver equals gs_shoot_batched + the FP64 update
    p + (-step) g (product rounded, then the sum), bit for bit."""
    ws = [inputs.make("slab", n, 90 + n, T=4, sigma=2.0) for n in (500, 320)]
    off = np.zeros(3, np.int64)
    off[1:] = np.cumsum([w.N for w in ws])
    cat = lambda k: dt(np.concatenate([getattr(w, k) for w in ws]))
    q0, X = cat("q0"), cat("X")
    p0 = torch.zeros_like(q0)
    step, iters = 1e-3, 5
    p, Eh = gs.descend_batched(q0, p0, X, off, 2.0, 4, 1.0, step=step, iters=iters, mode=mode)
    assert torch.equal(p0, torch.zeros_like(q0))  # the input is not modified
    pm = p0.clone()
    for it in range(iters):
        E, g = gs.shoot_batched(q0, pm, X, off, 2.0, 4, 1.0, mode=mode)
        assert torch.equal(Eh[it], E), it
        pm = pm + (-step) * g
    assert torch.equal(p, pm)
    tot = npy(Eh)[:, :, 0]
    assert np.all(np.diff(tot, axis=0) < 0), tot  # energy decreases for each subject
