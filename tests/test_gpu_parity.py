"""GPU path vs the FP64 oracle, element by element, through the C ABI
(Naess & Louis 2013, Sec. II: derivative maps, deflection, Eq. 4 Taylor sum, R).

Tolerances: FP64 mode <= 1e-6 relative RMS is the target; the kernels and the
oracle evaluate the same sums in a different order, so they agree to ~1e-12.
Mixed FP32 mode: <= 1e-4 relative RMS."""
import numpy as np
import pytest
import torch

import oracle.healpix as hp
import oracle.lens as OL
from gpu_util import max_rel, rel_rms, sky, to_dev

pytestmark = pytest.mark.gpu

api = pytest.importorskip("paper_1307_0719_gb300.api")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.mark.parametrize("nside,lmax,order", [(1, 2, 2), (2, 5, 3), (8, 16, 4), (16, 48, 6), (32, 64, 2)])
def test_synth_derivs_spin0_fp64(nside, lmax, order):
    s = sky(nside, lmax, pol=False, seeds=(5, 0, 1))
    ref = OL.derivative_maps(nside, lmax, order, alm_T=s["T"])["T"]
    out = api.synth_derivs(nside, lmax, order, to_dev(s)["T"], 0, api.FP64).cpu().numpy()
    for i in range(ref.shape[0]):
        assert rel_rms(out[i], ref[i]) < 1e-11, (i, rel_rms(out[i], ref[i]))


@pytest.mark.parametrize("nside,lmax,order", [(2, 5, 2), (8, 16, 4), (16, 40, 5)])
def test_synth_derivs_spin2_fp64(nside, lmax, order):
    s = sky(nside, lmax, pol=True, seeds=(5, 6, 1), b_scale=0.7)
    ref = OL.derivative_maps(nside, lmax, order, alm_E=s["E"], alm_B=s["B"])
    d = to_dev(s)
    eb = torch.cat([d["E"], d["B"]])
    out = api.synth_derivs(nside, lmax, order, eb, 2, api.FP64).cpu().numpy()
    K = ref["Q"].shape[0]
    for i in range(K):
        assert rel_rms(out[i], ref["Q"][i]) < 1e-11, ("Q", i)
        assert rel_rms(out[K + i], ref["U"][i]) < 1e-11, ("U", i)


def test_deflection_fp64():
    nside, lmax = 32, 64
    s = sky(nside, lmax, pol=False)
    a_th, a_ph = OL.deflection(nside, lmax, s["phi"])
    out = api.deflection(nside, lmax, to_dev(s)["phi"], api.FP64).cpu().numpy()
    assert rel_rms(out[0], a_th) < 1e-12
    assert rel_rms(out[1], a_ph) < 1e-12


@pytest.mark.parametrize("nside,lmax,order", [(16, 32, 3), (32, 64, 4), (64, 128, 0), (4, 12, 6)])
def test_lens_tqu_fp64(nside, lmax, order):
    s = sky(nside, lmax, pol=True, b_scale=0.4)
    ref = OL.lens(nside, lmax, order, s["T"], s["E"], s["B"], s["phi"], return_aux=True)
    d = to_dev(s)
    out = api.lens(nside, lmax, order, d["T"], d["E"], d["B"], d["phi"], api.FP64).cpu().numpy()
    for i, f in enumerate("TQU"):
        assert rel_rms(out[i], ref[f]) < 1e-10, (f, rel_rms(out[i], ref[f]))


def test_lens_nside64_T_only_fp64_and_brute_force():
    """Nside 64, lmax 128, order 3, temperature only, FP64; also against direct
    Y_lm sums at the displaced positions (the exact remap the series approximates)."""
    nside, lmax, order = 64, 128, 3
    s = sky(nside, lmax, pol=False, seeds=(0, 0, 1))
    ref = OL.lens(nside, lmax, order, s["T"], alm_phi=s["phi"])["T"]
    d = to_dev(s)
    out = api.lens(nside, lmax, order, d["T"], alm_phi=d["phi"], precision=api.FP64).cpu().numpy()[0]
    assert rel_rms(out, ref) < 1e-12
    pix = np.random.default_rng(0).choice(hp.npix(nside), 2000, replace=False)
    ex = OL.lens_exact(nside, lmax, s["T"], alm_phi=s["phi"], pix=pix)["T"]
    assert rel_rms(out[pix], ex) < 5e-6


def test_zero_deflection_identity():
    nside, lmax, order = 16, 32, 4
    s = sky(nside, lmax, pol=True)
    d = to_dev(s)
    out = api.lens(nside, lmax, order, d["T"], d["E"], d["B"], None, api.FP64).cpu().numpy()
    base = OL.derivative_maps(nside, lmax, 0, s["T"], s["E"], s["B"])
    for i, f in enumerate("TQU"):
        assert rel_rms(out[i], base[f][0]) < 1e-12


@pytest.mark.parametrize("nside,lmax,order", [(32, 64, 4), (64, 128, 3)])
def test_lens_mixed_fp32(nside, lmax, order):
    s = sky(nside, lmax, pol=True, b_scale=0.4)
    ref = OL.lens(nside, lmax, order, s["T"], s["E"], s["B"], s["phi"])
    d = to_dev(s)
    out = api.lens(nside, lmax, order, d["T"], d["E"], d["B"], d["phi"], api.MIXED_FP32).cpu().numpy()
    for i, f in enumerate("TQU"):
        assert rel_rms(out[i], ref[f]) < 1e-4, (f, rel_rms(out[i], ref[f]))


@pytest.mark.parametrize("precision,tol", [(api.MIXED_TF32x3, 1e-4), (api.MIXED_BF16x3, 1e-4), (api.MIXED_TF32, 5e-3)])
@pytest.mark.parametrize("nside,lmax,order", [(32, 64, 4), (64, 128, 3), (16, 40, 1), (128, 203, 2), (16, 40, 5),
                                               (8, 21, 6)])
def test_lens_tensor_core_forms(nside, lmax, order, precision, tol):
    """Contraction on the tensor cores: 3xTF32 and BF16x3 meet the mixed-precision
    target, plain TF32 is reported with its own (looser) bound."""
    s = sky(nside, lmax, pol=True, b_scale=0.4)
    ref = OL.lens(nside, lmax, order, s["T"], s["E"], s["B"], s["phi"])
    d = to_dev(s)
    out = api.lens(nside, lmax, order, d["T"], d["E"], d["B"], d["phi"], precision).cpu().numpy()
    for i, f in enumerate("TQU"):
        assert rel_rms(out[i], ref[f]) < tol, (f, rel_rms(out[i], ref[f]))


@pytest.mark.parametrize("precision,order", [(api.MIXED_TF32x3, 4), (api.MIXED_TF32x3, 5), (api.MIXED_BF16x3, 4),
                                             (api.MIXED_BF16x3, 6), (api.MIXED_FP32, 4), (api.FP64, 4)])
def test_lens_batch_equals_single_calls(precision, order):
    """tl_lens_batch over 20 realisations (on tensor-core plans groups of tl_plan_batch
    that share one basis, then the rest) gives what twenty tl_lens calls give."""
    nside, lmax = 32, 64
    skies = [to_dev(sky(nside, lmax, pol=True, seeds=(10 + i, 20 + i, 30 + i), b_scale=0.3)) for i in range(20)]
    plan = api.Plan(nside, lmax, order, pol=True, precision=precision)
    try:
        outs = [o.cpu().numpy() for o in plan.lens_batch(skies)]
        singles = [plan.lens(sk["T"], sk["E"], sk["B"], sk["phi"]).cpu().numpy() for sk in skies]
    finally:
        torch.cuda.synchronize()
        plan.close()
    tol = 1e-13 if precision == api.FP64 else 1e-6
    for o, s1 in zip(outs, singles):
        for i in range(3):
            assert rel_rms(o[i], s1[i]) <= tol


@pytest.mark.parametrize("precision", [api.MIXED_BF16x3, api.FP64])
def test_lens_batch_host_equals_device_call(precision):
    """tl_lens_batch_host (host buffers, copies inside the call) over 18 realisations,
    i.e. a full chunk of tl_plan_batch and a partial one, gives exactly the maps of
    tl_lens_batch on device buffers; a second, smaller call reuses the staging."""
    nside, lmax, order = 32, 64, 4
    host = [{k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
             sky(nside, lmax, pol=True, seeds=(80 + i, 90 + i, 100 + i), b_scale=0.3).items()} for i in range(18)]
    plan = api.Plan(nside, lmax, order, pol=True, precision=precision)
    try:
        dev = [{k: v.cuda() for k, v in h.items()} for h in host]
        ref = [o.cpu().numpy() for o in plan.lens_batch(dev)]
        got = [o.numpy() for o in plan.lens_batch_host(host)]
        got2 = [o.numpy() for o in plan.lens_batch_host(host[:3])]
    finally:
        torch.cuda.synchronize()
        plan.close()
    for r, g in zip(ref, got):
        assert np.array_equal(r, g)
    for r, g in zip(ref[:3], got2):
        assert np.array_equal(r, g)


def test_plan_batch_and_launch_count():
    """tl_plan_batch: 16 realisations per Legendre launch on the tensor-core forms up to
    order 5, 8 at order 6, 1 otherwise; tl_plan_batch_launches matches the kernels a
    tl_lens_batch call launches (counted by the CUDA profiler when it is available)."""
    plans = {(api.MIXED_TF32x3, 4): 16, (api.MIXED_TF32x3, 6): 8, (api.MIXED_BF16x3, 5): 16, (api.MIXED_BF16x3, 6): 8,
             (api.MIXED_FP32, 4): 1, (api.FP64, 3): 1}
    for (prec, order), want in plans.items():
        p = api.Plan(16, 32, order, pol=True, precision=prec)
        try:
            assert p.batch == want, (prec, order, p.batch)
        finally:
            p.close()
    nside, lmax, order = 32, 64, 4
    skies = [to_dev(sky(nside, lmax, pol=True, seeds=(50 + i, 60 + i, 70 + i), b_scale=0.3)) for i in range(18)]
    plan = api.Plan(nside, lmax, order, pol=True, precision=api.MIXED_TF32x3)
    try:
        plan.lens_batch(skies)  # warm: plan-time work is done
        torch.cuda.synchronize()
        from torch.profiler import ProfilerActivity, profile
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            plan.lens_batch(skies)
            torch.cuda.synchronize()
        names = [e.name for e in prof.events() if e.device_type.name == "CUDA"]
        ours = [n for n in names if any(k in n for k in ("ringfft", "legendre", "gather", "tcprep"))]
        if not ours:
            pytest.skip("the CUDA profiler recorded no kernels here")
        assert len(ours) == plan.batch_launches(18), (len(ours), plan.batch_launches(18))
    finally:
        torch.cuda.synchronize()
        plan.close()


def test_fp64_nside512_lmax1024_order4_vs_oracle_and_reruns():
    """The plain FP64 form at Nside 512, lmax 1024, order 4, T+Q/U (Sec. II, Eq. 4,
    R of Eq. 2): within 1e-6 of the oracle at every pixel of the cap-inclusive sample
    (relative to the map's RMS over the sample), and bit-for-bit equal over reruns."""
    import skygen
    w = skygen.WORKLOADS["nside512_lmax1024_n4_TQU"]
    s = skygen.make_sky(w.nside, w.lmax, w.pol, w.seed_t, w.seed_e, w.seed_phi, w.damp_t, w.damp_e)
    d = to_dev(s)
    plan = api.Plan(w.nside, w.lmax, w.order, pol=True, precision=api.FP64)
    try:
        runs = [plan.lens(d["T"], d["E"], d["B"], d["phi"]).cpu().numpy() for _ in range(3)]
    finally:
        torch.cuda.synchronize()
        plan.close()
    for r in runs[1:]:
        assert np.array_equal(r, runs[0])
    pix = hp.check_pixels(w.nside)
    ref = OL.lens_at_pixels(w.nside, w.lmax, w.order, pix, s["T"], s["E"], s["B"], s["phi"])
    for i, f in enumerate("TQU"):
        got = runs[0][i][pix]
        assert rel_rms(got, ref[f]) < 1e-6 and max_rel(got, ref[f]) < 1e-6, (f, rel_rms(got, ref[f]),
                                                                              max_rel(got, ref[f]))


@pytest.mark.parametrize("naive,at_pixel", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("precision,tol", [("FP64", 1e-10), ("MIXED_FP32", 1e-4), ("MIXED_BF16x3", 1e-4)])
def test_lens_geometry_options_vs_oracle(naive, at_pixel, precision, tol):
    """Plan flags TL_NAIVE (x' by coordinate addition, Sec. II.A) and
    TL_EXPAND_AT_PIXEL (the plain Taylor series about the output pixel itself, Sec. I
    Eq. 3a) against the oracle with the same options. The deflections are scaled up
    (about 75 arcmin RMS at Nside 32) so that expansion pixels move, the float path
    defers many pixels to its double pass, and naive addition carries points across
    the poles."""
    nside, lmax, order = 32, 64, 4
    s = sky(nside, lmax, pol=True, b_scale=0.4)
    phi = s["phi"] * 30.0
    ref = OL.lens(nside, lmax, order, s["T"], s["E"], s["B"], phi, naive=naive, at_pixel=at_pixel)
    d = to_dev(s)
    plan = api.Plan(nside, lmax, order, pol=True, precision=getattr(api, precision), naive=naive,
                    expand_at_pixel=at_pixel)
    try:
        out = plan.lens(d["T"], d["E"], d["B"], torch.from_numpy(phi).to("cuda:0")).cpu().numpy()
    finally:
        torch.cuda.synchronize()
        plan.close()
    for i, f in enumerate("TQU"):
        assert rel_rms(out[i], ref[f]) < tol, (f, rel_rms(out[i], ref[f]))


def test_adjoint_refuses_geometry_options():
    from paper_1307_0719_gb300 import _lib
    nside, lmax = 8, 16
    s = to_dev(sky(nside, lmax, pol=True, b_scale=0.3))
    plan = api.Plan(nside, lmax, 2, pol=True, precision=api.FP64, naive=True)
    try:
        g = torch.zeros(12 * nside * nside, dtype=torch.float64, device="cuda:0")
        with pytest.raises(_lib.TaylensError) as e:
            plan.lens_adjoint(s["T"], s["E"], s["B"], s["phi"], g, g, g)
        assert e.value.status == _lib.TL_ERR_UNSUPPORTED
    finally:
        torch.cuda.synchronize()
        plan.close()


@pytest.mark.parametrize("precision,tol", [("FP64", 1e-10), ("MIXED_FP32", 1e-4), ("MIXED_BF16x3", 1e-4)])
def test_lens_with_own_lmax_phi_vs_oracle(precision, tol):
    """The potential at its own band limit, the paper's min(8 Nside, 10000) (Sec. II.A):
    single calls, a batch (on the tensor-core forms: the realisations' Legendre launch
    without the potential, alpha from the deflection plan per realisation) and the
    deflection alone, against the oracle at the same lmax_phi; lmax_phi = lmax again
    restores the plain plan."""
    import skygen
    nside, lmax, order = 16, 32, 3
    lp = 8 * nside
    s = sky(nside, lmax, pol=True, b_scale=0.4)
    phi = skygen.make_sky(nside, lp, False, 0, 0, 5)["phi"] * 3.0
    ref = OL.lens(nside, lmax, order, s["T"], s["E"], s["B"], phi, lmax_phi=lp)
    a_th, a_ph = OL.deflection(nside, lp, phi)
    d = to_dev(s)
    dphi = torch.from_numpy(phi).cuda()
    plan = api.Plan(nside, lmax, order, pol=True, precision=getattr(api, precision), lmax_phi=lp)
    try:
        one = plan.lens(d["T"], d["E"], d["B"], dphi).cpu().numpy()
        two = plan.lens_batch([dict(T=d["T"], E=d["E"], B=d["B"], phi=dphi)] * 2)
        al = plan.deflection(dphi).cpu().numpy()
        plan.set_lmax_phi(lmax)
        back = plan.lens(d["T"], d["E"], d["B"], d["phi"]).cpu().numpy()
    finally:
        torch.cuda.synchronize()
        plan.close()
    for i, f in enumerate("TQU"):
        assert rel_rms(one[i], ref[f]) < tol, (f, rel_rms(one[i], ref[f]))
        for o in two:
            assert rel_rms(o[i].cpu().numpy(), ref[f]) < tol, (f, "batch")
    assert rel_rms(al[0], a_th) < tol and rel_rms(al[1], a_ph) < tol
    plain = OL.lens(nside, lmax, order, s["T"], s["E"], s["B"], s["phi"])
    for i, f in enumerate("TQU"):
        assert rel_rms(back[i], plain[f]) < tol, (f, "lmax_phi reset")


def test_lmax_phi_host_call_and_adjoint_refusal():
    """The host-buffer batch call stages the potential at its own coefficient count;
    the adjoint is refused while a separate lmax_phi is set."""
    import skygen
    nside, lmax, lp = 16, 32, 80
    s = sky(nside, lmax, pol=True, b_scale=0.4)
    phi = skygen.make_sky(nside, lp, False, 0, 0, 6)["phi"] * 3.0
    plan = api.Plan(nside, lmax, 2, pol=True, precision=api.MIXED_FP32, lmax_phi=lp)
    try:
        d = to_dev(s)
        dphi = torch.from_numpy(phi).cuda()
        dev = plan.lens(d["T"], d["E"], d["B"], dphi).cpu().numpy()
        host = plan.lens_batch_host([{k: torch.from_numpy(v) for k, v in
                                      dict(T=s["T"], E=s["E"], B=s["B"], phi=phi).items()}])[0].numpy()
        assert np.array_equal(dev, host)
        g = torch.ones(plan.npix, device="cuda", dtype=plan.dtype)
        with pytest.raises(api._lib.TaylensError) as ei:
            plan.lens_adjoint(d["T"], d["E"], d["B"], dphi, g, g, g)
        assert ei.value.status == api._lib.TL_ERR_UNSUPPORTED
    finally:
        torch.cuda.synchronize()
        plan.close()


@pytest.mark.parametrize("lmax_phi", [None, 80])
def test_batch_host_overlapped_copies_equal_device_call(lmax_phi):
    """The host-buffer batch call on a tensor-core plan (several realisations: the
    potential's and E/B's coefficients arrive on the copy stream while the temperature's
    Legendre launch runs, and each realisation's maps go back as soon as its gather has
    run) gives the device call's maps bit for bit, also with the potential's own band
    limit (its deflection plan reads the coefficients that arrive last)."""
    import skygen
    nside, lmax = 16, 32
    lp = lmax if lmax_phi is None else lmax_phi
    skies = []
    for i in range(3):
        s = sky(nside, lmax, pol=True, seeds=(30 + i, 40 + i, 1), b_scale=0.4)
        s["phi"] = skygen.make_sky(nside, lp, False, 0, 0, 50 + i)["phi"] * 3.0
        skies.append(s)
    plan = api.Plan(nside, lmax, 3, pol=True, precision=api.MIXED_BF16x3, lmax_phi=lmax_phi)
    try:
        dev = plan.lens_batch([to_dev(s) for s in skies])
        dev = [o.cpu().numpy() for o in dev]
        host = plan.lens_batch_host([{k: torch.from_numpy(v) for k, v in s.items()} for s in skies])
    finally:
        torch.cuda.synchronize()
        plan.close()
    for a, b in zip(dev, host):
        assert np.array_equal(a, b.numpy())
