"""The full-size workload in the launch configuration that bench.py times: Nside 2048,
lmax 4096, order 4, T+Q/U, the BF16x3 tensor-core contraction, sixteen realisations in
one tl_lens_batch call (one Legendre launch per field). Sampled output pixels are
compared with the FP64 oracle, which evaluates each of them on its own (the deflection
on the pixel's ring, the derivative values at its expansion pixel from direct Fourier
sums; Sec. II, Eq. 4 and the rotation R of Eq. 2). The sample includes the first and
last pixels (polar caps), the first and last pixels of the equatorial belt and the
equator. Tolerances: the mixed-precision target, 1e-4 relative RMS per map, and 3e-4
for the largest error relative to the sample's RMS. Collected last (file name): it
allocates about 100 GB and runs the oracle for tens of seconds."""
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


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def test_full_size_sampled_pixels_vs_oracle():
    w = skygen.WORKLOADS["nside2048_lmax4096_n4_TQU"]
    n = w.nside
    plan = api.Plan(w.nside, w.lmax, w.order, pol=w.pol, precision=api.MIXED_BF16x3)
    try:
        nb = plan.batch
        assert nb == 16
        # two distinct skies (the bench's first two realisations), repeated to fill the launch
        skies = [skygen.make_sky(w.nside, w.lmax, w.pol, w.seed_t + 100 * i, w.seed_e + 100 * i,
                                 w.seed_phi + 100 * i, w.damp_t, w.damp_e) for i in range(2)]
        dev = [to_dev(s) for s in skies]
        outs = plan.lens_batch([dev[i % 2] for i in range(nb)])
        torch.cuda.synchronize()
        maps = [o.cpu().numpy() for o in outs[:4]]
        del outs
    finally:
        torch.cuda.synchronize()
        plan.close()
    # copies of one sky in other columns of the same launch give the same maps
    for i in (2, 3):
        for f in range(3):
            assert rel_rms(maps[i][f], maps[i - 2][f]) <= 1e-6, (i, f)
    npix = hp.npix(n)
    edges = [0, 3, npix - 1, 2 * n * (n - 1), 2 * n * (n - 1) + 4 * n - 1, npix // 2,
             npix - 2 * n * (n - 1) - 1]
    rng = np.random.default_rng(11)
    pix = np.unique(np.concatenate([edges, rng.choice(npix, 9, replace=False)]))
    for i, sk in enumerate(skies):
        ref = OL.lens_at_pixels(w.nside, w.lmax, w.order, pix, sk["T"], sk["E"], sk["B"], sk["phi"],
                                nthreads=os.cpu_count())
        for f, name in enumerate("TQU"):
            got = maps[i][f][pix]
            assert rel_rms(got, ref[name]) < 1e-4, (i, name, rel_rms(got, ref[name]))
            assert max_rel(got, ref[name]) < 3e-4, (i, name, max_rel(got, ref[name]))
