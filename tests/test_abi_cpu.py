"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every entry point declared in include/gs.h, and argument errors
are rejected before any CUDA work."""
import ctypes
import os

import pytest

from paper_1907_04834_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1907_04834_gb300 import native
    native.build()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    names = _lib.declared_symbols()
    assert {"gs_create", "gs_destroy", "gs_shoot", "gs_shoot_grad", "gs_shoot_batched",
            "gs_last_error", "gs_sync", "gs_rhs", "gs_adj_rhs", "gs_tree"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_null_context_is_invalid(lib):
    prm = _lib.make_params(1.0, 4)
    assert lib.gs_shoot(None, None, None, 10, ctypes.byref(prm), None, None, None, None) == 1
    assert lib.gs_shoot_grad(None, None, None, None, 10, ctypes.byref(prm), None, None, None,
                             None) == 1
    assert lib.gs_sync(None, None) == 1
    assert lib.gs_last_error(None) == b"no context"


def test_create_rejects_bad_device(lib):
    h = ctypes.c_void_p()
    assert lib.gs_create(-1, ctypes.byref(h)) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_create(10 ** 6, ctypes.byref(h)) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_create(0, None) == _lib.GS_ERR_INVALID_ARG


def test_params_layout_matches_header(tmp_path):
    """The ctypes mirror of gs_params has the header's size and field
    offsets (a C program compiled against include/gs.h prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = ["sigma", "lambda", "thresh_sigmas", "T", "mode", "ckpt_every", "flags", "leaf_size",
             "criterion", "sympl_iters", "reserved"]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"gs.h\"\n"
                   "int main(void) { printf(\"%zu\", sizeof(gs_params));"
                   + "".join(f' printf(" %zu", offsetof(gs_params, {n}));' for n in names)
                   + " return 0; }\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    fields = ["sigma", "lambda_", "thresh_sigmas", "T", "mode", "ckpt_every", "flags", "leaf_size",
              "criterion", "sympl_iters", "reserved"]
    assert vals[0] == ctypes.sizeof(_lib.Params)
    assert vals[1:] == [getattr(_lib.Params, f).offset for f in fields]
    p = _lib.make_params(2.0, 7, "bh", 0.5, 3.0, 2)
    assert (p.sigma, p.lambda_, p.thresh_sigmas, p.T, p.mode, p.ckpt_every) == (
        2.0, 0.5, 3.0, 7, 1, 2)
