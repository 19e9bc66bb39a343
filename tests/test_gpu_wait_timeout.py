"""The bounded waits of the tensor-core Legendre kernels. With the self-test of
tl_plan_set_wait_limit the compute warps withhold their barrier arrivals, so the
issuing warp's wait for the tiles runs out after a short poll limit: the kernel
records the plan's error flag, waits (bounded) for its own MMAs, frees its tensor
memory and returns. tl_plan_device_error then reports TL_ERR_TIMEOUT (and clears
the flag), and once the plan is back to normal the same plan lenses correctly.
Nothing faults or hangs: every wait is bounded."""
import pytest
import torch

import oracle.lens as OL
from gpu_util import rel_rms, sky, to_dev

pytestmark = pytest.mark.gpu

_lib = pytest.importorskip("paper_1307_0719_gb300._lib")
api = pytest.importorskip("paper_1307_0719_gb300.api")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.mark.parametrize("precision", ["MIXED_BF16x3", "MIXED_TF32x3"])
def test_wait_timeout_is_reported_and_plan_recovers(precision):
    nside, lmax, order = 8, 16, 2
    s = sky(nside, lmax, pol=True, b_scale=0.3)
    d = to_dev(s)
    L = _lib.lib()
    plan = api.Plan(nside, lmax, order, pol=True, precision=getattr(api, precision))
    h = plan._h
    try:
        assert L.tl_plan_device_error(h) == _lib.TL_OK
        assert L.tl_plan_set_wait_limit(h, 4096, 1) == _lib.TL_OK
        plan.lens(d["T"], d["E"], d["B"], d["phi"])
        assert L.tl_plan_device_error(h) == _lib.TL_ERR_TIMEOUT
        assert L.tl_plan_device_error(h) == _lib.TL_OK  # cleared by the read
        assert L.tl_plan_set_wait_limit(h, 0, 0) == _lib.TL_OK
        out = plan.lens(d["T"], d["E"], d["B"], d["phi"]).cpu().numpy()
        assert L.tl_plan_device_error(h) == _lib.TL_OK
    finally:
        torch.cuda.synchronize()
        plan.close()
    ref = OL.lens(nside, lmax, order, s["T"], s["E"], s["B"], s["phi"])
    for i, f in enumerate("TQU"):
        assert rel_rms(out[i], ref[f]) < 1e-4, (f, rel_rms(out[i], ref[f]))
