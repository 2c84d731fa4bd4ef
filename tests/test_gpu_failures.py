"""Failure detection on the GPU without a fault: a bounded device-side wait
that cannot complete gives up and reports GS_ERR_TIMEOUT through the status
word; non-finite results are reported as GS_ERR_NONFINITE (a NaN input, and
semi-implicit passes that diverge); after each the context keeps working.

A call with device outputs is asynchronous, so its status arrives at the next
gs_sync; a call with host outputs returns finished results and its own
status.  Both routes are exercised."""
import numpy as np
import pytest
import torch

import paper_1907_04834_gb300 as gs
from paper_1907_04834_gb300 import inputs
from paper_1907_04834_gb300._lib import GS_ERR_NONFINITE, GS_ERR_TIMEOUT
from gpu_util import dt, npy

pytestmark = pytest.mark.gpu


def _still_works(oracle):
    w = inputs.make("slab", 400, 3, T=3)
    q1, _, _ = gs.shoot(dt(w.q0), dt(w.p0), w.sigma, w.T)
    q1o, _, _ = oracle.shoot(w.q0, w.p0, w.sigma, w.T)
    assert np.abs(npy(q1) - q1o).max() <= 1e-5 * w.sigma


def test_bounded_wait_times_out_and_context_survives(oracle):
    for _ in range(2):
        with pytest.raises(gs.GSError) as ei:
            gs.selftest_timeout()
        assert ei.value.status == GS_ERR_TIMEOUT
    _still_works(oracle)


def _shoot_status(q, p, sigma, T, on_host, **kw):
    """Run gs_shoot and return the GSError it reports (None when none)."""
    try:
        if on_host:
            gs.shoot(torch.from_numpy(q), torch.from_numpy(p), sigma, T, **kw)
        else:
            qd = dt(q)
            gs.shoot(qd, dt(p), sigma, T, **kw)
            gs.context(qd.device.index).sync()
    except gs.GSError as e:
        return e
    return None


@pytest.mark.parametrize("mode,on_host", [("exact", False), ("exact", True), ("bh", False),
                                          ("bh", True)])
def test_nan_input_reported(oracle, mode, on_host):
    w = inputs.make("blobs", 600, 4, T=3)
    p = w.p0.copy()
    p[17, 1] = np.nan
    e = _shoot_status(w.q0, p, w.sigma, w.T, on_host, mode=mode)
    assert e is not None and e.status == GS_ERR_NONFINITE
    _still_works(oracle)


def test_diverging_fixed_point_passes_reported(oracle):
    """Semi-implicit passes on a step too large for the fixed-point iteration
    to contract (200 points, momenta of about 4 sigma per unit time, T = 100,
    eight passes): the iterates blow up and the call reports it."""
    rng = np.random.default_rng(1)
    q = rng.normal(scale=2.0, size=(200, 3))
    p = rng.normal(scale=4.0, size=(200, 3))
    _, _, Ho = oracle.shoot_sympl(q, p, 1.0, 100, 8)
    assert not np.isfinite(Ho).all()  # the oracle diverges on this cloud too
    e = _shoot_status(q, p, 1.0, 100, False, sympl_iters=8, with_H=True)
    assert e is not None and e.status == GS_ERR_NONFINITE
    _still_works(oracle)
