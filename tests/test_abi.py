"""C ABI checks that need no GPU: the library loads, exports every function
include/lqcd.h declares, and validates arguments before touching a device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lqcd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lqcd_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1103_1363_gb300 import _build
    _build.build()
    from paper_1103_1363_gb300 import lqcd
    return lqcd


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "lqcd_dslash" in names and "lqcd_solve" in names
    for n in names:
        assert hasattr(lib._lib, n), n
    assert set(names) == set(lib.EXPORTED)


def test_create_validates_arguments(lib):
    with pytest.raises(lib.LqcdError) as e:
        lib.lqcd_create((4, 4, 3, 4))  # odd extent
    assert e.value.status == 1
    with pytest.raises(lib.LqcdError):
        lib.lqcd_create((4, 4, 4, 4), recon=8)
    with pytest.raises(lib.LqcdError):
        lib.lqcd_create((4, 4, 4, 4), max_nrhs=0)


def test_workspace_size_and_field_bytes(lib):
    cfg = lib.lqcd_config()
    for i, d in enumerate((4, 4, 4, 8)):
        cfg.dims[i] = d
    cfg.t_antiperiodic, cfg.recon, cfg.prec_mask, cfg.max_nrhs, cfg.gcr_nkrylov = 1, 12, 0xF, 2, 0
    ctx = C.c_void_p()
    assert lib._lib.lqcd_create(C.byref(cfg), None, C.byref(ctx)) == 0
    n = C.c_size_t()
    assert lib._lib.lqcd_workspace_size(ctx, C.byref(n)) == 0
    assert n.value > 0 and n.value % 256 == 0
    fb = C.c_size_t()
    assert lib._lib.lqcd_field_bytes(ctx, 1, C.byref(fb)) == 0
    assert fb.value == 256 * 96  # Vh = 256 sites (stride 256), 96 bytes per FP32 site
    # calls that need a workspace fail cleanly before one is set
    assert lib._lib.lqcd_gauge_load(ctx, None) != 0
    assert lib._lib.lqcd_dslash(ctx, None, None, 0, 0.1, 0.0, 0, 1, 1) == 3  # ERR_NOMEM: no workspace
    assert "workspace" in lib.lqcd_last_error()
    assert lib._lib.lqcd_destroy(ctx) == 0
