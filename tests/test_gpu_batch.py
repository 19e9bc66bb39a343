"""Batched lensing of realisations of uneven size (tl_batch_*): the persistent
launch and its CUDA-graph replay give what one tl_lens call per realisation gives,
and one realisation agrees with the FP64 oracle (Naess & Louis 2013, Eq. 4 + R)."""
import numpy as np
import pytest
import torch

import oracle.lens as OL
from gpu_util import rel_rms, sky, to_dev

pytestmark = pytest.mark.gpu
api = pytest.importorskip("paper_1307_0719_gb300.api")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


# groups: (8, 16) x 18, (16, 40) x 2, (32, 64), (32, 100): two waves of up to sixteen per group
NSIDES = [8, 16, 8, 32, 16, 8, 32] + [8] * 15
LMAXS = [16, 40, 16, 64, 40, 16, 100] + [16] * 15


def _skies():
    return [to_dev(sky(ns, lm, pol=True, seeds=(200 + i, 300 + i, 400 + i), b_scale=0.3))
            for i, (ns, lm) in enumerate(zip(NSIDES, LMAXS))]


@pytest.mark.parametrize("order,precision", [(3, "MIXED_TF32x3"), (5, "MIXED_TF32x3"), (4, "MIXED_BF16x3")])
def test_batch_modes_agree_and_match_oracle(order, precision):
    b = api.Batch(NSIDES, LMAXS, order, pol=True, precision=getattr(api, precision))
    try:
        assert b.groups == 4 and b.waves == 2
        skies = _skies()
        res = {}
        for mode in ("loop", "persistent", "graph", "graph"):
            outs = b.outputs()
            b.lens(skies, outs, mode)
            torch.cuda.synchronize()
            res.setdefault(mode, []).append([o.cpu().numpy() for o in outs])
        for mode in ("persistent", "graph"):
            for run in res[mode]:
                for i in range(len(NSIDES)):
                    for f in range(3):
                        assert rel_rms(run[i][f], res["loop"][0][i][f]) < 1e-6, (mode, i, f)
        i = 3
        ref = OL.lens(NSIDES[i], LMAXS[i], order, *(skies[i][k].cpu().numpy() for k in ("T", "E", "B", "phi")))
        for f, name in enumerate("TQU"):
            assert rel_rms(res["graph"][1][i][f], ref[name]) < 1e-4
    finally:
        torch.cuda.synchronize()
        b.close()


def test_batch_autotune_keeps_results():
    order = 2
    b = api.Batch(NSIDES[:4], LMAXS[:4], order, pol=True, precision=api.MIXED_TF32x3)
    try:
        skies = _skies()[:4]
        outs = b.outputs()
        b.lens(skies, outs, "loop")
        ref = [o.cpu().numpy() for o in outs]
        outs2 = b.outputs()
        b.autotune(skies, outs2)
        assert b.grid > 0
        b.lens(skies, outs2, "graph")
        torch.cuda.synchronize()
        for o, r in zip(outs2, ref):
            for f in range(3):
                assert rel_rms(o[f].cpu().numpy(), r[f]) < 1e-6
    finally:
        torch.cuda.synchronize()
        b.close()


def test_batch_uneven_nside256_to_2048_vs_oracle():
    """Uneven realisations at the sizes of a production mix (Nside 256 to 2048, lmax from
    2 to 2 Nside, order 4, the default BF16x3 form): the persistent launch and its graph
    replay against the per-realisation loop on every map, and realisations of each size
    against the FP64 oracle on sampled pixels (the first and last ring, the cap and belt
    edges and the equator, random pixels), to the mixed forms' 1e-4."""
    import os
    import skygen
    import oracle.healpix as hp
    nsides = [2048, 256, 512, 1024, 256, 512, 256]
    lmaxs = [4096, 512, 1024, 2048, 512, 768, 600]
    order = 4
    skies = [skygen.make_sky(ns, lm, True, 600 + i, 700 + i, 800 + i, 100.0, 800.0, b_scale=0.3)
             for i, (ns, lm) in enumerate(zip(nsides, lmaxs))]
    dev = [to_dev(s) for s in skies]
    b = api.Batch(nsides, lmaxs, order, pol=True, precision=api.MIXED_BF16x3)
    try:
        res = {}
        for mode in ("loop", "graph", "graph"):
            outs = b.outputs()
            b.lens(dev, outs, mode)
            torch.cuda.synchronize()
            res.setdefault(mode, []).append([o.cpu().numpy() for o in outs])
            del outs
    finally:
        torch.cuda.synchronize()
        b.close()
    for run in res["graph"]:
        for i in range(len(nsides)):
            for f in range(3):
                assert rel_rms(run[i][f], res["loop"][0][i][f]) < 1e-6, (i, f)
    for i in (0, 1, 2, 3):
        ns = nsides[i]
        pix = hp.check_pixels(ns, n_random=16, per_ring=8, cap_rings=1)
        sk = skies[i]
        ref = OL.lens_at_pixels(ns, lmaxs[i], order, pix, sk["T"], sk["E"], sk["B"], sk["phi"],
                                nthreads=os.cpu_count())
        for f, name in enumerate("TQU"):
            got = res["graph"][1][i][f][pix]
            assert rel_rms(got, ref[name]) < 1e-4, (ns, name, rel_rms(got, ref[name]))
