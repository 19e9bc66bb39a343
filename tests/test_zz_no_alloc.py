"""tl_deflection_noalloc: the deflection for callers that cannot allocate device
memory while they run. It must give what tl_deflection gives, on consecutive calls
that share its fixed device array. Collected last on purpose (file name), so a
run that stops at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import rel_rms, sky, to_dev

pytestmark = pytest.mark.gpu

_lib = pytest.importorskip("paper_1307_0719_gb300._lib")
api = pytest.importorskip("paper_1307_0719_gb300.api")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _noalloc(nside, lmax, precision, alm_phi, dtype):
    L = _lib.lib()
    npix = 12 * nside * nside
    out = torch.empty((2, npix), dtype=dtype, device="cuda")
    a = torch.view_as_real(alm_phi)
    st = L.tl_deflection_noalloc(nside, lmax, precision, ctypes.c_void_p(a.data_ptr()),
                                 ctypes.c_void_p(out[0].data_ptr()), ctypes.c_void_p(out[1].data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(st, "tl_deflection_noalloc")
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("precision,tol", [(_lib.TL_FP64, 1e-12), (_lib.TL_MIXED_FP32, 1e-6)])
@pytest.mark.parametrize("nside,lmax", [(32, 64), (128, 256)])
def test_noalloc_matches_tl_deflection_on_consecutive_calls(nside, lmax, precision, tol):
    dtype = torch.float64 if precision == _lib.TL_FP64 else torch.float32
    plan = api.Plan(nside, lmax, 1, pol=False, precision=precision)
    try:
        for seed in (11, 12):  # two calls in a row, different inputs
            s = to_dev(sky(nside, lmax, pol=False, seeds=(0, 0, seed)))
            ref = plan.deflection(s["phi"]).cpu().numpy()
            got = _noalloc(nside, lmax, precision, s["phi"], dtype)
            for i in range(2):
                assert rel_rms(got[i], ref[i]) < tol, (seed, i, rel_rms(got[i], ref[i]))
    finally:
        torch.cuda.synchronize()
        plan.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    L = _lib.lib()
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(z.data_ptr())
    assert L.tl_deflection_noalloc(256, 256, _lib.TL_FP64, p, p, p, None) == _lib.TL_ERR_ARG
    assert L.tl_deflection_noalloc(128, 300, _lib.TL_FP64, p, p, p, None) == _lib.TL_ERR_ARG


def test_noalloc_size_change_queued_behind_earlier_call_on_nonblocking_stream():
    """Two calls of different sizes queued on one non-blocking stream with no
    synchronisation between them: the second call lays the array out again and
    must first wait for the first call's kernels, which still read it."""
    sizes = [(32, 64), (128, 256)]
    refs, ins = [], []
    for nside, lmax in sizes:
        plan = api.Plan(nside, lmax, 1, pol=False, precision=_lib.TL_FP64)
        try:
            s = to_dev(sky(nside, lmax, pol=False, seeds=(0, 0, 21)))
            refs.append(plan.deflection(s["phi"]).cpu().numpy())
            ins.append(torch.view_as_real(s["phi"]))
        finally:
            torch.cuda.synchronize()
            plan.close()
    outs = [torch.empty((2, 12 * n * n), dtype=torch.float64, device="cuda") for n, _ in sizes]
    stream = torch.cuda.Stream()  # torch's pooled streams are non-blocking
    torch.cuda.synchronize()
    L = _lib.lib()
    for (nside, lmax), a, o in zip(sizes, ins, outs):
        st = L.tl_deflection_noalloc(nside, lmax, _lib.TL_FP64, ctypes.c_void_p(a.data_ptr()),
                                     ctypes.c_void_p(o[0].data_ptr()), ctypes.c_void_p(o[1].data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
        _lib.check(st, "tl_deflection_noalloc")
    stream.synchronize()
    for ref, o in zip(refs, outs):
        got = o.cpu().numpy()
        for i in range(2):
            assert rel_rms(got[i], ref[i]) < 1e-12, (i, rel_rms(got[i], ref[i]))
