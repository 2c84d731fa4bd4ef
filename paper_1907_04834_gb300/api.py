"""Python face of libgs: tensors in, tensors out, one C-ABI call each.

Inputs are float64 ``(N, 3)`` tensors, on a CUDA device (outputs are then
allocated there and the call is asynchronous on the current stream) or on
the CPU (the library stages them and the call returns finished results).
"""
from __future__ import annotations

import ctypes
import threading

import torch

from . import _lib
from ._lib import GS_BH, GS_EXACT, GSError, make_params

_ctxs: dict[int, "Context"] = {}
_lock = threading.Lock()


class Context:
    """A libgs context (workspace + device status) bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        st = self.lib.gs_create(int(device), ctypes.byref(h))
        if st != 0:
            raise GSError(st, f"gs_create(device={device}) failed")
        self.handle = h
        self.device = int(device)

    def check(self, st: int):
        if st != 0:
            raise GSError(st, self.lib.gs_last_error(self.handle).decode())

    def sync(self, stream=None):
        self.check(self.lib.gs_sync(self.handle, _stream_ptr(self.device, stream)))

    def close(self):
        if self.handle:
            self.lib.gs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def context(device: int | None = None) -> Context:
    if device is None:
        device = torch.cuda.current_device() if torch.cuda.is_available() else 0
    with _lock:
        if device not in _ctxs:
            _ctxs[device] = Context(device)
        return _ctxs[device]


def _stream_ptr(device, stream=None):
    if not torch.cuda.is_available():
        return None
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


def _pts(t, name, n=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(t)
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64 (got {t.dtype})")
    if t.dim() != 2 or t.shape[1] != 3:
        raise ValueError(f"{name} must have shape (N, 3) (got {tuple(t.shape)})")
    if n is not None and t.shape[0] != n:
        raise ValueError(f"{name} has {t.shape[0]} rows, expected {n}")
    return t.contiguous()


def _device_of(t: torch.Tensor) -> int | None:
    return t.device.index if t.is_cuda else None


def _like(t: torch.Tensor, shape=None) -> torch.Tensor:
    """Output buffer beside input t (pinned host memory for pinned inputs)."""
    shape = tuple(t.shape) if shape is None else shape
    if not t.is_cuda and t.is_pinned():
        return torch.empty(shape, dtype=torch.float64, pin_memory=True)
    return torch.empty(shape, dtype=torch.float64, device=t.device)


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _ctx_for(t: torch.Tensor) -> Context:
    d = _device_of(t)
    return context(d if d is not None else None)


def shoot(q0, p0, sigma, T, mode="exact", thresh=3.0, with_H=False, leaf_size=1, criterion=0,
          sympl_iters=0, stream=None):
    """Geodesic shooting (Eq. 1; explicit Euler, or with sympl_iters = M > 0
    the semi-implicit symplectic Euler step of M fixed-point passes).  Returns
    (q1, p1, H) with H = None or the tensor [H(q0,p0), H(q1,p1)]."""
    q0 = _pts(q0, "q0")
    p0 = _pts(p0, "p0", q0.shape[0])
    c = _ctx_for(q0)
    prm = make_params(sigma, T, mode, 0.0, thresh, leaf_size=leaf_size, criterion=criterion,
                      sympl_iters=sympl_iters)
    q1, p1 = _like(q0), _like(q0)
    H = _like(q0, (2,)) if with_H else None
    c.check(c.lib.gs_shoot(c.handle, _ptr(q0), _ptr(p0), q0.shape[0], ctypes.byref(prm), _ptr(q1),
                           _ptr(p1), _ptr(H), _stream_ptr(c.device, stream)))
    return q1, p1, H


def shoot_grad(q0, p0, X, sigma, T, lam=1.0, mode="exact", thresh=3.0, ckpt_every=0,
               leaf_size=1, criterion=0, sympl_iters=0, stream=None):
    """Objective of Eq. 2 and dE/dp0 (sympl_iters = M > 0: of the
    semi-implicit scheme with M fixed-point passes per step).  Returns
    (E, grad, q1) with E = [E, H(q0,p0), lambda |q1 - X|^2]."""
    q0 = _pts(q0, "q0")
    n = q0.shape[0]
    p0, X = _pts(p0, "p0", n), _pts(X, "X", n)
    c = _ctx_for(q0)
    prm = make_params(sigma, T, mode, lam, thresh, ckpt_every, leaf_size=leaf_size,
                      criterion=criterion, sympl_iters=sympl_iters)
    E = _like(q0, (3,))
    grad, q1 = _like(q0), _like(q0)
    c.check(c.lib.gs_shoot_grad(c.handle, _ptr(q0), _ptr(p0), _ptr(X), n, ctypes.byref(prm),
                                _ptr(E), _ptr(grad), _ptr(q1), _stream_ptr(c.device, stream)))
    return E, grad, q1


def shoot_batched(q0, p0, X, offsets, sigma, T, lam=1.0, mode="exact", thresh=3.0,
                  ckpt_every=0, leaf_size=1, criterion=0, stream=None):
    """Independent registrations of the subjects delimited by ``offsets``
    (S+1 increasing ints, rows of q0/p0/X).  Returns (E (S, 3), grad (N, 3)),
    E[s] = [E, H(q0,p0), lambda |q1 - X|^2] of subject s."""
    q0 = _pts(q0, "q0")
    n = q0.shape[0]
    p0, X = _pts(p0, "p0", n), _pts(X, "X", n)
    off = torch.as_tensor(offsets, dtype=torch.int64).cpu().contiguous()
    S = off.numel() - 1
    if S < 1 or int(off[-1]) != n:
        raise ValueError("offsets must have S+1 entries ending at N")
    c = _ctx_for(q0)
    prm = make_params(sigma, T, mode, lam, thresh, ckpt_every, leaf_size=leaf_size, criterion=criterion)
    E = _like(q0, (S, 3))
    grad = _like(q0)
    c.check(c.lib.gs_shoot_batched(c.handle, S, _ptr(off), _ptr(q0), _ptr(p0), _ptr(X),
                                   ctypes.byref(prm), _ptr(E), _ptr(grad),
                                   _stream_ptr(c.device, stream)))
    return E, grad


def descend_batched(q0, p0, X, offsets, sigma, T, lam=1.0, step=0.1, iters=50, mode="exact",
                    thresh=3.0, ckpt_every=0, leaf_size=1, criterion=0, stream=None):
    """Fixed-step gradient descent on the subjects' initial momenta
    (gs_descend_batched): ``iters`` times p0 <- p0 - step * dE/dp0.
    Returns (p0 after the last update (N, 3), E history (iters, S, 3))."""
    q0 = _pts(q0, "q0")
    n = q0.shape[0]
    p0, X = _pts(p0, "p0", n), _pts(X, "X", n)
    off = torch.as_tensor(offsets, dtype=torch.int64).cpu().contiguous()
    S = off.numel() - 1
    if S < 1 or int(off[-1]) != n:
        raise ValueError("offsets must have S+1 entries ending at N")
    c = _ctx_for(q0)
    prm = make_params(sigma, T, mode, lam, thresh, ckpt_every, leaf_size=leaf_size, criterion=criterion)
    p = p0.clone()
    Eh = _like(q0, (int(iters), S, 3))
    c.check(c.lib.gs_descend_batched(c.handle, S, _ptr(off), _ptr(q0), _ptr(p), _ptr(X),
                                     ctypes.byref(prm), float(step), int(iters), _ptr(Eh),
                                     _stream_ptr(c.device, stream)))
    return p, Eh


def lbfgs(q0, p0, X, sigma, T, lam=1.0, m=8, iters=50, gtol=1e-6, mode="exact", thresh=3.0,
          ckpt_every=0, leaf_size=1, criterion=0, stream=None):
    """L-BFGS on the initial momenta (gs_lbfgs).  Returns (p0 after the last
    iterate, E history of the initial point and each accepted iterate,
    iterations done)."""
    q0 = _pts(q0, "q0")
    n = q0.shape[0]
    p0, X = _pts(p0, "p0", n), _pts(X, "X", n)
    c = _ctx_for(q0)
    prm = make_params(sigma, T, mode, lam, thresh, ckpt_every, leaf_size=leaf_size, criterion=criterion)
    p = p0.clone()
    Eh = torch.empty(int(iters) + 1, dtype=torch.float64)
    done = ctypes.c_int32(0)
    c.check(c.lib.gs_lbfgs(c.handle, _ptr(q0), _ptr(p), _ptr(X), n, ctypes.byref(prm), int(m),
                           int(iters), float(gtol), _ptr(Eh), ctypes.byref(done),
                           _stream_ptr(c.device, stream)))
    return p, Eh[: done.value + 1], done.value


def autotune(q, p, sigma, thresh=3.0, candidates=(1, 2, 4, 8, 16, 32), stream=None):
    """Barnes-Hut leaf size that runs one forward + adjoint right-hand side
    fastest on state (q, p) (gs_autotune).  Returns (best, {leaf: ms})."""
    q = _pts(q, "q")
    n = q.shape[0]
    p = _pts(p, "p", n)
    c = _ctx_for(q)
    prm = make_params(sigma, 1, "bh", 0.0, thresh)
    cand = (ctypes.c_int32 * len(candidates))(*[int(v) for v in candidates])
    ms = (ctypes.c_double * len(candidates))()
    best = ctypes.c_int32(0)
    c.check(c.lib.gs_autotune(c.handle, _ptr(q), _ptr(p), n, ctypes.byref(prm), cand,
                              len(candidates), ctypes.byref(best), ms,
                              _stream_ptr(c.device, stream)))
    return best.value, {int(v): ms[k] for k, v in enumerate(candidates)}


def autotune_exact(q, p, sigma, candidates=(1, 2, 3, 4, 6, 8, 12, 16, 24, 32), stream=None):
    """Source splits J of the exact forward and adjoint kernels that run one
    right-hand side each fastest on state (q, p) (gs_autotune_exact).
    Returns ((J_fwd, J_adj), {J: (fwd ms, adj ms)}); apply with
    set_option("exact_splits_fwd", J_fwd) and set_option("exact_splits_adj", J_adj)."""
    q = _pts(q, "q")
    n = q.shape[0]
    p = _pts(p, "p", n)
    c = _ctx_for(q)
    prm = make_params(sigma, 1, "exact", 0.0)
    cand = (ctypes.c_int32 * len(candidates))(*[int(v) for v in candidates])
    ms = (ctypes.c_double * (2 * len(candidates)))()
    best = (ctypes.c_int32 * 2)()
    c.check(c.lib.gs_autotune_exact(c.handle, _ptr(q), _ptr(p), n, ctypes.byref(prm), cand,
                                    len(candidates), best, ms, _stream_ptr(c.device, stream)))
    return (best[0], best[1]), {int(v): (ms[2 * k], ms[2 * k + 1])
                                for k, v in enumerate(candidates)}


def flow(q0, p0, x0, sigma, T, mode="exact", thresh=3.0, leaf_size=1, criterion=0,
         stream=None):
    """Shooting that carries tracer points x0 (M, 3) through the velocity
    field of Eq. 3 (gs_flow; mode "exact" or "bh").  Returns (q1, p1, x1)."""
    q0 = _pts(q0, "q0")
    n = q0.shape[0]
    p0 = _pts(p0, "p0", n)
    x0 = _pts(x0, "x0")
    m = x0.shape[0]
    c = _ctx_for(q0)
    prm = make_params(sigma, T, mode, 0.0, thresh, leaf_size=leaf_size, criterion=criterion)
    q1, p1, x1 = _like(q0), _like(q0), _like(x0)
    c.check(c.lib.gs_flow(c.handle, _ptr(q0), _ptr(p0), n, _ptr(x0) if m else None, m,
                          ctypes.byref(prm), _ptr(q1), _ptr(p1), _ptr(x1) if m else None,
                          _stream_ptr(c.device, stream)))
    return q1, p1, x1


def velocity(q, p, x, sigma, mode="exact", thresh=3.0, leaf_size=1, criterion=0, stream=None):
    """Velocity field of Eq. 3 at points x (M, 3): v = sum_i G(|x - q_i|) p_i
    (mode "bh": Barnes-Hut over the particles' tree)."""
    q = _pts(q, "q")
    n = q.shape[0]
    p = _pts(p, "p", n)
    x = _pts(x, "x")
    c = _ctx_for(q)
    v = _like(x)
    prm = make_params(sigma, 1, mode, 0.0, thresh, leaf_size=leaf_size, criterion=criterion)
    c.check(c.lib.gs_velocity(c.handle, _ptr(q), _ptr(p), n, _ptr(x), x.shape[0],
                              ctypes.byref(prm), _ptr(v), _stream_ptr(c.device, stream)))
    return v


def rhs(q, p, sigma, mode="exact", thresh=3.0, leaf_size=1, criterion=0, with_counts=True,
        stream=None):
    """One forward right-hand side: (F, Phi, (point pairs, node pairs)), or
    (F, Phi) with with_counts=False (no counts requested: the lean walk)."""
    q = _pts(q, "q")
    p = _pts(p, "p", q.shape[0])
    c = _ctx_for(q)
    prm = make_params(sigma, 1, mode, 0.0, thresh, leaf_size=leaf_size, criterion=criterion)
    F, Phi = torch.empty_like(q), torch.empty_like(q)
    cnt = (ctypes.c_int64 * 2)()
    c.check(c.lib.gs_rhs(c.handle, _ptr(q), _ptr(p), q.shape[0], ctypes.byref(prm), _ptr(F),
                         _ptr(Phi), cnt if with_counts else None, _stream_ptr(c.device, stream)))
    return (F, Phi, (cnt[0], cnt[1])) if with_counts else (F, Phi)


def adj_rhs(q, p, al, be, sigma, mode="exact", thresh=3.0, leaf_size=1, criterion=0,
            with_counts=True, stream=None):
    """One adjoint right-hand side: (dA, dB, counts), or (dA, dB) with
    with_counts=False."""
    q = _pts(q, "q")
    n = q.shape[0]
    p, al, be = _pts(p, "p", n), _pts(al, "al", n), _pts(be, "be", n)
    c = _ctx_for(q)
    prm = make_params(sigma, 1, mode, 0.0, thresh, leaf_size=leaf_size, criterion=criterion)
    dA, dB = torch.empty_like(q), torch.empty_like(q)
    cnt = (ctypes.c_int64 * 2)()
    c.check(c.lib.gs_adj_rhs(c.handle, _ptr(q), _ptr(p), _ptr(al), _ptr(be), n,
                             ctypes.byref(prm), _ptr(dA), _ptr(dB), cnt if with_counts else None,
                             _stream_ptr(c.device, stream)))
    return (dA, dB, (cnt[0], cnt[1])) if with_counts else (dA, dB)


def tree(q, stream=None):
    """The octree the Barnes-Hut steps build on q: dict with ``codes`` (N,)
    Morton codes, ``order`` (N,), ``nodes`` (M, 4) {depth, first, count,
    skip} in preorder (depth -1 = single-point leaf), ``range`` (M, 6)."""
    q = _pts(q, "q")
    n = q.shape[0]
    c = _ctx_for(q)
    cap = 2 * n + 8
    dev = q.device
    codes = torch.empty(n, dtype=torch.int32, device=dev)
    order = torch.empty(n, dtype=torch.int32, device=dev)
    nodes = torch.empty((cap, 4), dtype=torch.int32, device=dev)
    rng = torch.empty((cap, 6), dtype=torch.float32, device=dev)
    m = ctypes.c_int64()
    c.check(c.lib.gs_tree(c.handle, _ptr(q), n, _ptr(codes), _ptr(order), _ptr(nodes), _ptr(rng),
                          cap, ctypes.byref(m), _stream_ptr(c.device, stream)))
    M = m.value
    return dict(codes=codes, order=order, nodes=nodes[:M], range=rng[:M], n_nodes=M)


def shoot_traj(q0, p0, sigma, T, mode="exact", thresh=3.0, leaf_size=1, criterion=0,
               sympl_iters=0, stream=None):
    """Shooting that returns the discrete path (gs_shoot_traj): (qtraj, ptraj),
    each (T + 1, N, 3), state k = after k steps."""
    q0 = _pts(q0, "q0")
    n = q0.shape[0]
    p0 = _pts(p0, "p0", n)
    c = _ctx_for(q0)
    prm = make_params(sigma, T, mode, 0.0, thresh, leaf_size=leaf_size, criterion=criterion,
                      sympl_iters=sympl_iters)
    qt, pt = _like(q0, (int(T) + 1, n, 3)), _like(q0, (int(T) + 1, n, 3))
    c.check(c.lib.gs_shoot_traj(c.handle, _ptr(q0), _ptr(p0), n, ctypes.byref(prm), _ptr(qt),
                                _ptr(pt), _stream_ptr(c.device, stream)))
    return qt, pt


def bh_tally(q, sigma, thresh=3.0, leaf_size=1, criterion=0, with_stats=False, stream=None):
    """Per-target record of the Barnes-Hut decisions on the tree of q
    (gs_bh_tally): int64 (N, 5) {point interactions, node interactions,
    fingerprint of the points, fingerprint of the nodes, nodes reached}; with
    with_stats also (walk iterations, list entries)."""
    q = _pts(q, "q")
    n = q.shape[0]
    c = _ctx_for(q)
    prm = make_params(sigma, 1, "bh", 0.0, thresh, leaf_size=leaf_size, criterion=criterion)
    out = torch.empty((n, 5), dtype=torch.int64, device=q.device)
    st = (ctypes.c_int64 * 2)()
    c.check(c.lib.gs_bh_tally(c.handle, _ptr(q), n, ctypes.byref(prm), _ptr(out),
                              st if with_stats else None, _stream_ptr(c.device, stream)))
    return (out, (st[0], st[1])) if with_stats else out


def tree_sums(q, p, al=None, be=None, stream=None):
    """Per-node sums {q, p, alpha, beta} (M, 12) of the octree of q in
    gs_tree's preorder (gs_tree_sums)."""
    q = _pts(q, "q")
    n = q.shape[0]
    p = _pts(p, "p", n)
    if (al is None) != (be is None):
        raise ValueError("al and be must both be given or both be None")
    if al is not None:
        al, be = _pts(al, "al", n), _pts(be, "be", n)
    c = _ctx_for(q)
    cap = 2 * n + 8
    sums = torch.empty((cap, 12), dtype=torch.float64, device=q.device)
    m = ctypes.c_int64()
    c.check(c.lib.gs_tree_sums(c.handle, _ptr(q), _ptr(p), _ptr(al), _ptr(be), n, _ptr(sums),
                               cap, ctypes.byref(m), _stream_ptr(c.device, stream)))
    return sums[: m.value]


def set_option(name: str, value: int, device: int | None = None):
    """Sets a tuning option of the device's context (see gs_set_option)."""
    c = context(device)
    c.check(c.lib.gs_set_option(c.handle, name.encode(), int(value)))


def selftest_timeout(device: int | None = None, stream=None):
    """Failure-detection self-test (gs_selftest_timeout): a device-side
    bounded wait that cannot complete must give up and report GS_ERR_TIMEOUT;
    raises GSError with that status when it does."""
    c = context(device)
    c.check(c.lib.gs_selftest_timeout(c.handle, _stream_ptr(c.device, stream)))


def timing(enable: bool = True, device: int | None = None):
    """Turns per-kernel-class event timing on or off (see gs_timing)."""
    c = context(device)
    c.check(c.lib.gs_timing(c.handle, int(bool(enable))))


def timing_read(device: int | None = None):
    """{class: (launch groups, ms)} since the last read, and the number of
    kernels the library launched meanwhile."""
    c = context(device)
    n = len(_lib.KERNEL_CLASSES)
    la = (ctypes.c_int64 * n)()
    ms = (ctypes.c_double * n)()
    tot = ctypes.c_int64()
    c.check(c.lib.gs_timing_read(c.handle, la, ms, ctypes.byref(tot)))
    return {k: (la[i], ms[i]) for i, k in enumerate(_lib.KERNEL_CLASSES)}, tot.value


def alu_peaks(device: int = 0):
    """Measured lane-op rates: (FP32 FMA, FP32 via f32x2 FMA, MUFU ex2) per s."""
    lib = _lib.load()
    out = (ctypes.c_double * 3)()
    st = lib.gs_alu_peaks(int(device), out)
    if st != 0:
        raise GSError(st, "gs_alu_peaks failed")
    return tuple(out)


class GeodesicShoot(torch.autograd.Function):
    """E(p0) of Eq. 2 as an autograd function of p0; the backward pass returns
    the adjoint gradient computed together with E."""

    @staticmethod
    def forward(ctx, p0, q0, X, sigma, T, lam, mode, thresh, ckpt_every):
        E, grad, _ = shoot_grad(q0, p0.detach(), X, sigma, T, lam, mode, thresh, ckpt_every)
        ctx.save_for_backward(grad)
        return E[0]

    @staticmethod
    def backward(ctx, gE):
        (grad,) = ctx.saved_tensors
        return gE * grad, None, None, None, None, None, None, None, None


def energy(p0, q0, X, sigma, T, lam=1.0, mode="exact", thresh=3.0, ckpt_every=0):
    """Differentiable registration objective E(p0) (Eq. 2)."""
    return GeodesicShoot.apply(p0, q0, X, sigma, T, lam, mode, thresh, ckpt_every)
