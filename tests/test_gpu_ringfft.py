"""Ring synthesis of the single-precision forms where the register-pass kernels run
(rings of 2^10 .. 2^13 pixels without aliasing: the belt at Nside 256 .. 2048; Bluestein
lengths 2048 and 4096 on the cap rings) and the shared-memory Bluestein of length 1024
beside them: the derivative maps d_theta^j d_phi^k of Eq. 4 against the oracle's
per-ring library FFT (Sec. II.B), over the whole sphere and over the belt alone, for band
limits below, at and above half the belt ring length, spin 0 and spin 2.

Tolerance: 5e-5 relative RMS per map and ring. The single-precision Legendre data
set the level: both ring-FFT kernels (register passes and shared memory) measure
the same errors ring by ring, up to 3.7e-5 on the d_phi maps of the last cap rings
at Nside 2048, which share a transform with the larger d_phi^0 map of their plane
(its rounding leaks in at float epsilon times the magnitude ratio). The target of
the mixed forms for the lensed maps is 1e-4."""
import numpy as np
import pytest
import torch

import oracle.healpix as hp
import oracle.lens as OL
from gpu_util import rel_rms, sky, to_dev

pytestmark = pytest.mark.gpu

api = pytest.importorskip("paper_1307_0719_gb300.api")
TOL = 5e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _belt(nside):
    ncap = 2 * nside * (nside - 1)
    return slice(ncap, hp.npix(nside) - ncap)


@pytest.mark.parametrize("nside,lmax,order", [(256, 511, 4), (256, 512, 3), (256, 700, 4), (512, 1024, 4)])
def test_synth_derivs_spin0_mixed_fp32(nside, lmax, order):
    s = sky(nside, lmax, pol=False, seeds=(7, 0, 1))
    ref = OL.derivative_maps(nside, lmax, order, alm_T=s["T"])["T"]
    out = api.synth_derivs(nside, lmax, order, to_dev(s)["T"], 0, api.MIXED_FP32).cpu().numpy()
    b = _belt(nside)
    for i in range(ref.shape[0]):
        assert rel_rms(out[i], ref[i]) < TOL, (i, rel_rms(out[i], ref[i]))
        assert rel_rms(out[i][b], ref[i][b]) < TOL, (i, "belt", rel_rms(out[i][b], ref[i][b]))


@pytest.mark.parametrize("nside,lmax,order", [(256, 512, 4), (256, 700, 2)])
def test_synth_derivs_spin2_mixed_fp32(nside, lmax, order):
    s = sky(nside, lmax, pol=True, seeds=(7, 8, 1), b_scale=0.6)
    ref = OL.derivative_maps(nside, lmax, order, alm_E=s["E"], alm_B=s["B"])
    d = to_dev(s)
    out = api.synth_derivs(nside, lmax, order, torch.cat([d["E"], d["B"]]), 2, api.MIXED_FP32).cpu().numpy()
    K = ref["Q"].shape[0]
    b = _belt(nside)
    for i in range(K):
        for f, o in (("Q", out[i]), ("U", out[K + i])):
            assert rel_rms(o, ref[f][i]) < TOL, (f, i, rel_rms(o, ref[f][i]))
            assert rel_rms(o[b], ref[f][i][b]) < TOL, (f, i, "belt")


def _rings_vs_oracle(nside, lmax, order, rings, spin, precision, tol):
    """Derivative maps on chosen rings (0-based ring index) against the oracle's
    ring coefficients and library-FFT ring synthesis on those rings alone."""
    import oracle.sht as sht
    tab = hp.ring_table(nside)
    jk = OL.derivative_pairs(order)
    if spin == 0:
        s = sky(nside, lmax, pol=False, seeds=(9, 0, 1))
        F = sht.ring_coeffs(lmax, order, tab["theta"][rings], alm_T=s["T"])
        fields = {"T": F["T"]}
        alm = to_dev(s)["T"]
    else:
        s = sky(nside, lmax, pol=True, seeds=(9, 10, 1), b_scale=0.5)
        F = sht.ring_coeffs(lmax, order, tab["theta"][rings], alm_E=s["E"], alm_B=s["B"])
        fields = {"Q": F["Q"], "U": F["U"]}
        d = to_dev(s)
        alm = torch.cat([d["E"], d["B"]])
    plan = api.Plan(nside, lmax, order, pol=(spin == 2), precision=precision)
    try:
        out = plan.synth_derivs(alm, spin)
        K = len(jk)
        for q, r in enumerate(rings):
            a, n = int(tab["first"][r]), int(tab["nphi"][r])
            got = out[:, a:a + n].cpu().numpy()
            for fi, (f, Fr) in enumerate(fields.items()):
                ref = OL.ring_synthesis(Fr[q], n, float(tab["phi0"][r]), jk)
                for i in range(K):
                    e = rel_rms(got[fi * K + i], ref[i])
                    assert e < tol, (r, n // 4, f, jk[i], e)
    finally:
        torch.cuda.synchronize()
        plan.close()


@pytest.mark.parametrize("spin", [0, 2])
def test_cap_rings_bluestein_2048_nside1024(spin):
    """Cap rings of 4 i pixels with i in 513 .. 1023 (Bluestein length 2048), the
    power-of-two ring i = 512, the last cap ring and a belt ring, north and south."""
    nside = 1024
    rings = [512, 600, 777, 1022, 1023, 2047, 4 * nside - 1 - 600]
    _rings_vs_oracle(nside, 2 * nside, 4, [r - 1 for r in rings], spin, api.MIXED_FP32, TOL)


def test_cap_rings_bluestein_4096_nside2048():
    """Cap rings with i in 1025 .. 2047 (Bluestein length 4096) and 513 .. 1023 (2048)
    at the full-size geometry, north and south, and a belt ring."""
    nside = 2048
    rings = [700, 1025, 1536, 2039, 2047, 4095, 4 * nside - 1 - 1300]
    _rings_vs_oracle(nside, 2 * nside, 4, [r - 1 for r in rings], 0, api.MIXED_FP32, TOL)


@pytest.mark.parametrize("spin", [0, 2])
def test_cap_rings_bluestein_1024_nside512(spin):
    """Cap rings with i in 257 .. 511 (Bluestein length 1024, shared-memory passes), the
    power-of-two ring i = 256 and the last cap ring, north and south, and a belt ring."""
    nside = 512
    rings = [256, 257, 300, 444, 511, 1024, 4 * nside - 1 - 300]
    _rings_vs_oracle(nside, 2 * nside, 4, [r - 1 for r in rings], spin, api.MIXED_FP32, TOL)
