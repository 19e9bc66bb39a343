"""The float gather's choice of expansion pixel, checked pixel by pixel against the
oracle (Naess & Louis 2013, Sec. II.B: x0' is the centre of the HEALPix pixel that
contains x').

At order 0 the Taylor sum of Eq. 4 is its leading term, so the lensed map is the
unlensed map read at the expansion pixel, T'(p) = T(q(p)). A plan expanding about
the output pixel itself (q = p) returns T with the same kernels, so the default
plan's output must equal that map read at the oracle's q, computed in FP64 from the
same single-precision deflection the kernels used. This is index work: the check is
exact, over every pixel of the map."""
import numpy as np
import pytest
import torch

import oracle.lens as OL
import oracle.healpix as hp
from gpu_util import sky

pytestmark = pytest.mark.gpu

api = pytest.importorskip("paper_1307_0719_gb300.api")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def oracle_cells(nside, a_th, a_ph, naive, chunk=1 << 21):
    """q(p) for every pixel from the oracle's displacement and ang2pix, in chunks."""
    tab = hp.ring_table(nside)
    npx = 12 * nside * nside
    q = np.empty(npx, dtype=np.int64)
    for lo in range(0, npx, chunk):
        pix = np.arange(lo, min(npx, lo + chunk))
        ring, j = hp.pix2ring(nside, pix)
        r = ring - 1
        z, s, th = tab["z"][r], tab["sint"][r], tab["theta"][r]
        ph = tab["phi0"][r] + 2.0 * np.pi * j / tab["nphi"][r]
        th2, ph2, z2, s2, _ = OL.target_point(th, z, s, ph, a_th[pix], a_ph[pix], naive=naive)
        q[pix], _, _ = OL.expansion_point(nside, pix, th2, ph2, z2, s2, th, ph)
    return q


@pytest.mark.parametrize("nside,lmax,scale,naive", [
    (1024, 2048, 4.0, False),   # deflections of a few pixels; polar pixels through the double pass
    (256, 512, 4.0, False),
    (256, 512, 4.0, True),      # naive coordinate addition (Sec. II.A)
    (64, 128, 20.0, False),     # deflections of many pixels, up to the 0.02 rad limit and beyond
])
def test_float_lookup_cells_equal_oracle_cells(nside, lmax, scale, naive):
    s = sky(nside, lmax, pol=False)
    T = torch.from_numpy(s["T"]).cuda()
    phi = torch.from_numpy(s["phi"] * scale).cuda()
    plan = api.Plan(nside, lmax, 0, pol=False, precision=api.MIXED_FP32, naive=naive)
    at = api.Plan(nside, lmax, 0, pol=False, precision=api.MIXED_FP32, naive=naive, expand_at_pixel=True)
    try:
        out = plan.lens(T, alm_phi=phi)[0].cpu().numpy()
        M = at.lens(T, alm_phi=phi)[0].cpu().numpy()
        al = plan.deflection(phi).cpu().numpy().astype(np.float64)
    finally:
        torch.cuda.synchronize()
        plan.close()
        at.close()
    q = oracle_cells(nside, al[0], al[1], naive)
    moved = np.count_nonzero(q != np.arange(q.size))
    assert moved > q.size // 20, moved  # the deflections move many pixels to another cell
    bad = np.flatnonzero(out != M[q])
    assert bad.size == 0, (bad.size, bad[:8], q[bad[:8]])
