"""gs_rhs_exact_noalloc -- the exact forward right-hand side for callers
that cannot allocate device memory (their device memory belongs to their own
pool allocator, or an allocation's implicit synchronisation is not
acceptable in their loop).  It must give the same F and Phi as gs_rhs, call
after call, through the C ABI, from one fixed scratch array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def _noalloc(lib, q, p, sigma, stream):
    F, Phi = torch.empty_like(q), torch.empty_like(q)
    st = lib.gs_rhs_exact_noalloc(ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                                  q.shape[0], float(sigma), ctypes.c_void_p(F.data_ptr()),
                                  ctypes.c_void_p(Phi.data_ptr()), ctypes.c_void_p(stream))
    return st, F, Phi


def _max_rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_noalloc_matches_rhs_twice_in_a_row():
    lib = _lib.load()
    stream = torch.cuda.current_stream(DEV).cuda_stream
    # two calls in a row on different clouds and sizes (the second sees the
    # first call's leftovers in the shared scratch), then the first again
    cases = [inputs.make("slab", 3001, 41), inputs.make("blobs", 1337, 42)]
    for w in cases + cases[:1]:
        q = torch.as_tensor(w.q0, dtype=torch.float64, device=DEV)
        p = torch.as_tensor(w.p0, dtype=torch.float64, device=DEV)
        F_ref, Phi_ref, _ = gs.rhs(q, p, w.sigma)
        st, F, Phi = _noalloc(lib, q, p, w.sigma, stream)
        assert st == 0
        torch.cuda.synchronize()
        assert _max_rel(F, F_ref) <= 1e-5
        assert _max_rel(Phi, Phi_ref) <= 1e-5


def test_noalloc_rejects_bad_requests():
    lib = _lib.load()
    stream = torch.cuda.current_stream(DEV).cuda_stream
    n = _lib.RHS_NOALLOC_MAX_N + 1
    q = torch.zeros((n, 3), dtype=torch.float64, device=DEV)
    st, _, _ = _noalloc(lib, q, q, 1.0, stream)
    assert st == _lib.GS_ERR_INVALID_ARG
    qh = torch.zeros((10, 3), dtype=torch.float64)  # host memory is refused
    F = torch.empty((10, 3), dtype=torch.float64, device=DEV)
    st = lib.gs_rhs_exact_noalloc(ctypes.c_void_p(qh.data_ptr()), ctypes.c_void_p(qh.data_ptr()),
                                  10, 1.0, ctypes.c_void_p(F.data_ptr()),
                                  ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(stream))
    assert st == _lib.GS_ERR_INVALID_ARG
