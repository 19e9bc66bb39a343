"""The C-ABI library loads without a GPU and exports every function include/taylens.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "taylens.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tl_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1307_0719_gb300 import build, _lib
    build.build()
    return _lib.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "tl_lens" in names and "tl_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_1307_0719_gb300 import _lib
    assert set(_declared()) == set(_lib.SIGNATURES)


def test_host_argument_checks(lib):
    from paper_1307_0719_gb300 import _lib as L
    h = ctypes.c_void_p()
    assert lib.tl_plan_create(3, 4, 1, 1, 0, 1, ctypes.byref(h)) == L.TL_ERR_ARG      # nside not 2^k
    assert lib.tl_plan_create(4, 33, 1, 1, 0, 1, ctypes.byref(h)) == L.TL_ERR_ARG     # lmax > 8 nside
    assert lib.tl_plan_create(4, 8, 7, 1, 0, 1, ctypes.byref(h)) == L.TL_ERR_ARG      # order > 6
    assert lib.tl_plan_create(4, 8, 2, 1, 9, 1, ctypes.byref(h)) == L.TL_ERR_ARG      # precision
    assert lib.tl_plan_create(4, 8, 2, L.TL_SPIN_QU, 0, 1, ctypes.byref(h)) == L.TL_ERR_UNSUPPORTED  # Q/U alone
    # every precision form passes the argument checks (without a GPU the CUDA set-up then fails)
    for prec in (L.TL_FP64, L.TL_MIXED_FP32, L.TL_MIXED_TF32, L.TL_MIXED_TF32x3, L.TL_MIXED_BF16x3):
        rc = lib.tl_plan_create(4, 8, 2, L.TL_SPIN_T | L.TL_SPIN_QU, prec, 1, ctypes.byref(h))
        assert rc in (L.TL_OK, L.TL_ERR_CUDA), (prec, rc)
        if rc == L.TL_OK:
            lib.tl_plan_destroy(h)
    assert lib.tl_plan_create(4, 8, 2, 1, 0, 8, ctypes.byref(h)) == L.TL_ERR_ARG      # unknown flag
    assert lib.tl_lens(None, None, None, None, None, None, None, None, None) == L.TL_ERR_ARG
    assert lib.tl_plan_destroy(None) == L.TL_OK
    assert lib.tl_plan_set_wait_limit(None, 0, 0) == L.TL_ERR_ARG
    assert lib.tl_plan_set_lmax_phi(None, 100) == L.TL_ERR_ARG
    assert lib.tl_lens_batch_host(None, 1, None, None, None, None, None, None, None, None) == L.TL_ERR_ARG
    assert lib.tl_plan_workspace_bytes(None) == 0
    assert lib.tl_status_string(L.TL_ERR_ARG) == b"invalid argument"
    # allocation-free entry point: sizes beyond its fixed array are refused up front
    assert lib.tl_deflection_noalloc(256, 256, 0, None, None, None, None) == L.TL_ERR_ARG


def test_analysis_argument_checks(lib):
    from paper_1307_0719_gb300 import _lib as L
    assert lib.tl_map2alm(None, None, None, None, None, None, None, None) == L.TL_ERR_ARG
    assert lib.tl_anafast(-1, None, None, None, None, None) == L.TL_ERR_ARG
    assert lib.tl_anafast(8, None, None, None, None, None) == L.TL_ERR_ARG
