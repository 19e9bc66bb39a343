"""The full-size workload: Nside 2048, lmax 4096, order 4, T+Q/U (Sec. II, Eq. 4 and
the rotation R of Eq. 2), in every precision form against the FP64 oracle on sampled
output pixels that the oracle evaluates one by one (the deflection on the pixel's
ring, the derivative values at its expansion pixel from direct Fourier sums).

The sample (oracle.healpix.check_pixels, 528 pixels) holds every pixel of the first
and last four rings, where the recurrence is least well conditioned, 64 pixels on the
last cap ring and the first belt ring of each hemisphere and on the equator, and 128
random pixels. The BF16x3 form runs in the launch configuration that bench.py times:
sixteen realisations in one tl_lens_batch call (one Legendre launch per field).

Tolerances (the targets of the mixed and FP64 forms, 1e-4 and 1e-6 relative RMS per
map), applied per pixel: every sampled pixel's error, relative to the RMS of the map
over the sample, must stay below the target, and so must the relative RMS over the
sample. Collected last (file name): it allocates about 100 GB and runs the oracle for
a minute or two per sky."""
import os

import numpy as np
import pytest
import torch

import oracle.healpix as hp
import oracle.lens as OL
import skygen
from gpu_util import max_rel, rel_rms, to_dev

pytestmark = pytest.mark.gpu

api = pytest.importorskip("paper_1307_0719_gb300.api")

W = skygen.WORKLOADS["nside2048_lmax4096_n4_TQU"]
MIXED_TOL = 1e-4
FP64_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.fixture(scope="module")
def skies():
    # the bench's first two realisations
    return [skygen.make_sky(W.nside, W.lmax, W.pol, W.seed_t + 100 * i, W.seed_e + 100 * i,
                            W.seed_phi + 100 * i, W.damp_t, W.damp_e) for i in range(2)]


@pytest.fixture(scope="module")
def pix():
    return hp.check_pixels(W.nside)


@pytest.fixture(scope="module")
def refs(skies, pix):
    return [OL.lens_at_pixels(W.nside, W.lmax, W.order, pix, sk["T"], sk["E"], sk["B"], sk["phi"],
                              nthreads=os.cpu_count()) for sk in skies]


def _check(maps, ref, pix, tol, what):
    for f, name in enumerate("TQU"):
        got = maps[f][pix]
        rr, mr = rel_rms(got, ref[name]), max_rel(got, ref[name])
        assert rr < tol and mr < tol, (what, name, rr, mr)


def _run(precision, skies, fill16):
    plan = api.Plan(W.nside, W.lmax, W.order, pol=W.pol, precision=precision)
    try:
        dev = [to_dev(s) for s in skies]
        if fill16:
            nb = plan.batch
            assert nb == 16
            outs = plan.lens_batch([dev[i % len(dev)] for i in range(nb)])
            torch.cuda.synchronize()
            maps = [o.cpu().numpy() for o in outs[:2 * len(dev)]]
        elif plan.batch > 1:
            outs = plan.lens_batch(dev)
            torch.cuda.synchronize()
            maps = [o.cpu().numpy() for o in outs]
        else:
            maps = []
            for d in dev:
                maps.append(plan.lens(d["T"], d["E"], d["B"], d["phi"]).cpu().numpy())
        del dev
    finally:
        torch.cuda.synchronize()
        plan.close()
    return maps


def test_full_size_bf16x3_batch16_vs_oracle(skies, pix, refs):
    maps = _run(api.MIXED_BF16x3, skies, fill16=True)
    # copies of one sky in other columns of the same launch give the same maps
    for i in (2, 3):
        for f in range(3):
            assert rel_rms(maps[i][f], maps[i - 2][f]) <= 1e-6, (i, f)
    for i, ref in enumerate(refs):
        _check(maps[i], ref, pix, MIXED_TOL, ("bf16x3", i))


@pytest.mark.parametrize("precision", ["MIXED_TF32x3", "MIXED_FP32"])
def test_full_size_mixed_forms_vs_oracle(precision, skies, pix, refs):
    maps = _run(getattr(api, precision), skies, fill16=False)
    for i, ref in enumerate(refs):
        _check(maps[i], ref, pix, MIXED_TOL, (precision, i))


def test_full_size_fp64_vs_oracle(skies, pix, refs):
    maps = _run(api.FP64, skies[:1], fill16=False)
    _check(maps[0], refs[0], pix, FP64_TOL, ("fp64", 0))
