"""gs_rhs_exact_noalloc -- the exact forward right-hand side for callers
that cannot allocate device memory (their device memory belongs to their own
pool allocator, or an allocation's implicit synchronisation is not
acceptable in their loop).  Through the C ABI it must give the oracle's F
and Phi within the right-hand-side tolerance, call after call from one
fixed scratch array, at the largest size it accepts (where the scratch is
fully used) and at sizes that are not a whole number of source tiles, and
it must not change the device's free memory.

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


def _call(lib, q, p, sigma, F, Phi, stream):
    return lib.gs_rhs_exact_noalloc(ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                                    q.shape[0], float(sigma), ctypes.c_void_p(F.data_ptr()),
                                    ctypes.c_void_p(Phi.data_ptr()), ctypes.c_void_p(stream))


def _max_rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_noalloc_matches_oracle_twice_in_a_row(oracle):
    lib = _lib.load()
    stream = torch.cuda.current_stream(DEV).cuda_stream
    # the largest accepted size, then sizes off the 512-source tiles; each
    # call sees the previous call's leftovers in the shared scratch; the
    # largest size comes back at the end
    cases = [inputs.make("slab", _lib.RHS_NOALLOC_MAX_N, 41), inputs.make("blobs", 1337, 42),
             inputs.make("ellipsoid", 5003, 43)]
    ref = {}
    for w in cases:
        F, Phi, _ = oracle.rhs(w.q0, w.p0, w.sigma)
        ref[w.N] = (F, Phi)
    for w in cases + cases[:1]:
        q = torch.as_tensor(w.q0, dtype=torch.float64, device=DEV)
        p = torch.as_tensor(w.p0, dtype=torch.float64, device=DEV)
        Fo, Phio = ref[w.N]
        for _ in range(2):
            F, Phi = torch.full_like(q, np.nan), torch.full_like(q, np.nan)
            assert _call(lib, q, p, w.sigma, F, Phi, stream) == 0
            torch.cuda.synchronize()
            eF, eP = _max_rel(F.cpu().numpy(), Fo), _max_rel(Phi.cpu().numpy(), Phio)
            assert eF <= 1e-5 and eP <= 1e-5, (w.N, eF, eP)
    print(f"\nno-alloc RHS at N={_lib.RHS_NOALLOC_MAX_N}, 1337, 5003 against the oracle: "
          f"within 1e-5")


def test_noalloc_allocates_nothing():
    """After a first call on the device (which loads the library's module
    and with it the fixed scratch), further calls leave the device's free
    memory unchanged."""
    lib = _lib.load()
    stream = torch.cuda.current_stream(DEV).cuda_stream
    w = inputs.make("blobs", 4000, 44)
    q = torch.as_tensor(w.q0, dtype=torch.float64, device=DEV)
    p = torch.as_tensor(w.p0, dtype=torch.float64, device=DEV)
    F, Phi = torch.empty_like(q), torch.empty_like(q)
    assert _call(lib, q, p, w.sigma, F, Phi, stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(DEV)
    reserved0 = torch.cuda.memory_reserved(DEV)
    for _ in range(3):
        assert _call(lib, q, p, w.sigma, F, Phi, stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(DEV)
    assert free1 == free0
    assert torch.cuda.memory_reserved(DEV) == reserved0


def test_noalloc_rejects_bad_requests():
    lib = _lib.load()
    stream = torch.cuda.current_stream(DEV).cuda_stream
    n = _lib.RHS_NOALLOC_MAX_N + 1
    q = torch.zeros((n, 3), dtype=torch.float64, device=DEV)
    assert _call(lib, q, q, 1.0, q, q, stream) == _lib.GS_ERR_INVALID_ARG
    qh = torch.zeros((10, 3), dtype=torch.float64)  # host memory is refused
    F = torch.empty((10, 3), dtype=torch.float64, device=DEV)
    assert _call(lib, qh, qh, 1.0, F, F, stream) == _lib.GS_ERR_INVALID_ARG
