"""GPU point-set geodesic shooting with the Barnes-Hut approximation
(arXiv 1907.04834) for sm_103a.

The computation lives in ``libgs.so`` (C ABI in ``include/gs.h``); the names
re-exported here are thin tensor wrappers around its entry points.  Importing
the package does not load CUDA; the first call does, and it fails loudly if
the library has not been built.
"""
_API = ("shoot", "shoot_grad", "shoot_batched", "descend_batched", "lbfgs", "autotune",
        "autotune_exact", "flow",
        "velocity",
        "rhs",
        "adj_rhs", "tree", "shoot_traj", "bh_tally", "tree_sums",
        "energy", "GeodesicShoot", "Context", "context", "GSError", "timing", "timing_read",
        "alu_peaks", "set_option", "selftest_timeout")


def __getattr__(name):
    if name in _API:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)


def build(force: bool = False, verbose: bool = False) -> str:
    from .native import build as _b
    return _b(force=force, verbose=verbose)
