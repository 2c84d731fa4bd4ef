"""FP64 CPU oracle for point-set geodesic shooting (arXiv 1907.04834).

TEST INFRASTRUCTURE ONLY.  This package is the plain reference the CUDA path
is checked against: ``gsref.c`` written from the paper (Sec. 2.1 Eq. 1-3 for
the exact flow and its adjoint, Sec. 2.2 for the octree and the three-case
traversal with the summaries of Eq. 4).  Only ``tests/``, the smoke check
and the benchmark's CPU-baseline leg may import it.  It shares no code with
the CUDA library and never imports it.

All arrays are float64 ``(N, 3)`` C-contiguous numpy arrays.  ``mode`` is
``0`` (exact all pairs) or ``1`` (Barnes-Hut with the ``thresh``-sigma rule).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsref.c")
_LIB = os.path.join(_HERE, "libgsref.so")

EXACT = 0
BH = 1
TRUNC = 2

_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``gsref.c`` into ``libgsref.so`` next to it (gcc, OpenMP, no
    floating-point contraction so the FP32 decision rule is reproducible)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    i64, dbl, cint = ctypes.c_int64, ctypes.c_double, ctypes.c_int
    lib.gsref_rhs.argtypes = [i64, _f64p, _f64p, dbl, cint, dbl, cint, cint, _f64p, _f64p,
                              _i64p]
    lib.gsref_rhs_rows.argtypes = [i64, _f64p, _f64p, dbl, i64, _i64p, _f64p, _f64p]
    lib.gsref_adj_rhs.argtypes = [i64, _f64p, _f64p, _f64p, _f64p, dbl, cint, dbl, cint, cint,
                                  _f64p, _f64p, _i64p]
    lib.gsref_adj_rhs_rows.argtypes = [i64, _f64p, _f64p, _f64p, _f64p, dbl, i64, _i64p,
                                       _f64p, _f64p]
    lib.gsref_shoot.argtypes = [i64, _f64p, _f64p, dbl, cint, cint, dbl, cint, cint, _f64p,
                                _f64p, _f64p]
    lib.gsref_shoot_rk4.argtypes = [i64, _f64p, _f64p, dbl, cint, _f64p, _f64p]
    lib.gsref_shoot_sympl.argtypes = [i64, _f64p, _f64p, dbl, cint, cint, dbl, cint, cint, cint,
                                      _f64p, _f64p, _f64p]
    lib.gsref_shoot_grad.argtypes = [i64, _f64p, _f64p, _f64p, dbl, cint, dbl, cint, dbl, cint,
                                     cint, _f64p, _f64p, _f64p]
    lib.gsref_morton.argtypes = [i64, _f64p, _u32p, _u32p]
    lib.gsref_velocity.argtypes = [i64, _f64p, _f64p, i64, _f64p, dbl, _f64p]
    lib.gsref_velocity_bh.argtypes = [i64, _f64p, _f64p, i64, _f64p, dbl, dbl, cint, cint, _f64p]
    lib.gsref_flow.argtypes = [i64, _f64p, _f64p, i64, _f64p, dbl, cint, cint, dbl, cint, cint,
                               _f64p, _f64p, _f64p]
    lib.gsref_tree.argtypes = [i64, _f64p, _f64p, ctypes.c_void_p, ctypes.c_void_p, _i64p, i64,
                               _i64p, _f64p, _f32p]
    lib.gsref_tree.restype = i64
    lib.gsref_bh_list.argtypes = [i64, _f64p, _f64p, dbl, dbl, cint, cint, i64, i64, _i64p,
                                  _i64p]
    lib.gsref_bh_list.restype = i64
    lib.gsref_shoot_grad_sympl.argtypes = [i64, _f64p, _f64p, _f64p, dbl, cint, dbl, cint, dbl,
                                           cint, cint, cint, _f64p, _f64p, _f64p]
    lib.gsref_bh_tally.argtypes = [i64, _f64p, dbl, dbl, cint, cint, _i64p]
    lib.gsref_num_threads.restype = cint
    _lib = lib
    return lib


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().gsref_num_threads())


def rhs(q, p, sigma, mode=EXACT, thresh=3.0, leaf=1, crit=0):
    """Forward right-hand side (F, Phi) of Eq. 1, plus interaction counts
    (point-point, point-node).  leaf > 1: Barnes-Hut leaf-size variant (a
    near node of at most `leaf` points is taken exactly); crit = 1:
    opening-angle variant of the far test with theta = thresh."""
    q, p = _c(q), _c(p)
    n = q.shape[0]
    F, Phi = np.empty_like(q), np.empty_like(q)
    cnt = np.zeros(2, np.int64)
    _load().gsref_rhs(n, q, p, float(sigma), int(mode), float(thresh), int(leaf), int(crit), F,
                      Phi, cnt)
    return F, Phi, cnt


def velocity(q, p, x, sigma, mode=EXACT, thresh=3.0, leaf=1, crit=0):
    """Velocity field of Eq. 3 at points x: v(x) = sum_i G(|x - q_i|) p_i
    (mode BH: Barnes-Hut over the particles' tree)."""
    q, p, x = _c(q), _c(p), _c(x)
    v = np.empty_like(x)
    if mode == BH:
        _load().gsref_velocity_bh(q.shape[0], q, p, x.shape[0], x, float(sigma), float(thresh),
                                  int(leaf), int(crit), v)
    else:
        _load().gsref_velocity(q.shape[0], q, p, x.shape[0], x, float(sigma), v)
    return v


def flow(q0, p0, x0, sigma, T, mode=EXACT, thresh=3.0, leaf=1, crit=0):
    """Shooting with tracer points x carried by Eq. 3's field (Euler steps in
    lockstep; mode EXACT or BH for both): returns q(1), p(1), x(1)."""
    q0, p0, x0 = _c(q0), _c(p0), _c(x0)
    q1, p1, x1 = np.empty_like(q0), np.empty_like(q0), np.empty_like(x0)
    _load().gsref_flow(q0.shape[0], q0, p0, x0.shape[0], x0, float(sigma), int(T), int(mode),
                       float(thresh), int(leaf), int(crit), q1, p1, x1)
    return q1, p1, x1


def rhs_rows(q, p, sigma, rows):
    """Exact F, Phi for the selected rows only."""
    q, p = _c(q), _c(p)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    F = np.empty((len(rows), 3))
    Phi = np.empty((len(rows), 3))
    _load().gsref_rhs_rows(q.shape[0], q, p, float(sigma), len(rows), rows, F, Phi)
    return F, Phi


def adj_rhs(q, p, al, be, sigma, mode=EXACT, thresh=3.0, leaf=1, crit=0):
    """Adjoint right-hand side: alpha^k = a + h dA, beta^k = b + h dB."""
    q, p, al, be = _c(q), _c(p), _c(al), _c(be)
    dA, dB = np.empty_like(q), np.empty_like(q)
    cnt = np.zeros(2, np.int64)
    _load().gsref_adj_rhs(q.shape[0], q, p, al, be, float(sigma), int(mode), float(thresh),
                          int(leaf), int(crit), dA, dB, cnt)
    return dA, dB, cnt


def adj_rhs_rows(q, p, al, be, sigma, rows):
    q, p, al, be = _c(q), _c(p), _c(al), _c(be)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    dA = np.empty((len(rows), 3))
    dB = np.empty((len(rows), 3))
    _load().gsref_adj_rhs_rows(q.shape[0], q, p, al, be, float(sigma), len(rows), rows, dA, dB)
    return dA, dB


def shoot(q0, p0, sigma, T, mode=EXACT, thresh=3.0, leaf=1, crit=0):
    """Geodesic shooting: returns q(1), p(1), [H(0), H(1)]."""
    q0, p0 = _c(q0), _c(p0)
    q1, p1 = np.empty_like(q0), np.empty_like(q0)
    H = np.zeros(2)
    _load().gsref_shoot(q0.shape[0], q0, p0, float(sigma), int(T), int(mode), float(thresh),
                        int(leaf), int(crit), q1, p1, H)
    return q1, p1, H


def shoot_rk4(q0, p0, sigma, T):
    """Exact-kernel shooting by classical RK4 (a check of the right-hand side,
    not a scheme of the method): q(1), p(1)."""
    q0, p0 = _c(q0), _c(p0)
    q1, p1 = np.empty_like(q0), np.empty_like(q0)
    _load().gsref_shoot_rk4(q0.shape[0], q0, p0, float(sigma), int(T), q1, p1)
    return q1, p1


def shoot_sympl(q0, p0, sigma, T, iters, mode=EXACT, thresh=3.0, leaf=1, crit=0):
    """Semi-implicit symplectic Euler shooting (gsref_shoot_sympl: `iters`
    fixed-point passes per step; 0 = explicit Euler): q(1), p(1), [H(0), H(1)]."""
    q0, p0 = _c(q0), _c(p0)
    q1, p1 = np.empty_like(q0), np.empty_like(q0)
    H = np.zeros(2)
    _load().gsref_shoot_sympl(q0.shape[0], q0, p0, float(sigma), int(T), int(mode),
                              float(thresh), int(leaf), int(crit), int(iters), q1, p1, H)
    return q1, p1, H


def shoot_grad(q0, p0, X, sigma, T, lam, mode=EXACT, thresh=3.0, leaf=1, crit=0):
    """Objective E = [total, H0, data] (Eq. 2) and dE/dp0 by the discrete
    adjoint; also returns q(1)."""
    q0, p0, X = _c(q0), _c(p0), _c(X)
    E = np.zeros(3)
    grad, q1 = np.empty_like(q0), np.empty_like(q0)
    _load().gsref_shoot_grad(q0.shape[0], q0, p0, X, float(sigma), int(T), float(lam),
                             int(mode), float(thresh), int(leaf), int(crit), E, grad, q1)
    return E, grad, q1


def shoot_grad_sympl(q0, p0, X, sigma, T, lam, iters, mode=EXACT, thresh=3.0, leaf=1, crit=0):
    """Objective (Eq. 2) and dE/dp0 for the semi-implicit scheme of
    shoot_sympl (`iters` fixed-point passes per step; 0 = shoot_grad), by
    the discrete adjoint of its step: (E, grad, q1)."""
    q0, p0, X = _c(q0), _c(p0), _c(X)
    E = np.zeros(3)
    grad, q1 = np.empty_like(q0), np.empty_like(q0)
    _load().gsref_shoot_grad_sympl(q0.shape[0], q0, p0, X, float(sigma), int(T), float(lam),
                                   int(mode), float(thresh), int(leaf), int(crit), int(iters),
                                   E, grad, q1)
    return E, grad, q1


def morton(q):
    """Quantised coordinates (N,3) uint32 and 30-bit Morton codes (N,)."""
    q = _c(q)
    kq = np.zeros((q.shape[0], 3), np.uint32)
    code = np.zeros(q.shape[0], np.uint32)
    _load().gsref_morton(q.shape[0], q, kq, code)
    return kq, code


def tree(q, p, al=None, be=None):
    """The paper's insertion octree, exported in DFS preorder.

    Returns a dict: ``order`` (DFS point order), ``depth``, ``leaf``, ``n``,
    ``first``, ``nchild`` (non-empty children), ``parent`` per node, FP64
    sums ``sq, sp, sa, sb`` (nodes, 3) and FP32 ranges ``lo, hi``."""
    q, p = _c(q), _c(p)
    n = q.shape[0]
    cap = 11 * n + 8
    order = np.zeros(n, np.int64)
    info = np.zeros((cap, 6), np.int64)
    stat = np.zeros((cap, 12))
    rng = np.zeros((cap, 6), np.float32)
    alc = _c(al) if al is not None else None
    bec = _c(be) if be is not None else None
    cnt = _load().gsref_tree(n, q, p,
                             alc.ctypes.data if alc is not None else None,
                             bec.ctypes.data if bec is not None else None,
                             order, cap, info, stat, rng)
    info, stat, rng = info[:cnt], stat[:cnt], rng[:cnt]
    return dict(order=order, depth=info[:, 0], leaf=info[:, 1], n=info[:, 2], first=info[:, 3],
                nchild=info[:, 4], parent=info[:, 5], sq=stat[:, 0:3], sp=stat[:, 3:6],
                sa=stat[:, 6:9], sb=stat[:, 9:12], lo=rng[:, 0:3], hi=rng[:, 3:6])


def bh_list(q, p, sigma, m, thresh=3.0, leaf=1, crit=0):
    """Interaction list of target ``m``: arrays (kind, id); kind 0 = point
    (id = point index), kind 1 = node summary (id = preorder node id)."""
    q, p = _c(q), _c(p)
    cap = q.shape[0] * 2 + 16
    kind = np.zeros(cap, np.int64)
    ids = np.zeros(cap, np.int64)
    L = _load().gsref_bh_list(q.shape[0], q, p, float(sigma), float(thresh), int(leaf),
                              int(crit), int(m), cap, kind, ids)
    return kind[:L], ids[:L]


def bh_tally(q, sigma, thresh=3.0, leaf=1, crit=0):
    """Per-target record of the Barnes-Hut decisions on the tree of q: an
    (N, 5) array {point interactions, node interactions, fingerprint of the
    points taken, fingerprint of the nodes summarised, nodes of >= 2 points
    reached}; the fingerprints are sums modulo 2**64 of splitmix64(key) over
    the sources, key = (DFS first position << 32) | member count (columns
    2-3 as uint64 bit patterns); a chain of single-child cells counts once."""
    q = _c(q)
    out = np.zeros((q.shape[0], 5), np.int64)
    _load().gsref_bh_tally(q.shape[0], q, float(sigma), float(thresh), int(leaf), int(crit), out)
    return out
