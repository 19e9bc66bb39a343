"""GPU adjoint (tl_lens_adjoint) against the FP64 oracle's adjoint, element by
element, plus identities that hold for the GPU path on its own: the dot-product
(transpose) identity for the unlensed fields, which enter linearly at fixed
deflection, and torch autograd through LensFunction.

Tolerances. T, E, B gradients depend on the forward only through the expansion
pixel, offsets and rotation angle, so FP64 agrees with the oracle to ~1e-12.
The phi and alpha gradients use the geometry Jacobian: exact (dual numbers) on
the GPU, Richardson central differences in the oracle (error ~1e-10 of each
Jacobian row's largest entry), hence 1e-8. Mixed forms (float recurrence in the difference form, double
accumulators): measured about 6e-7 relative RMS for T, E, B in FP32, 3xTF32 and BF16x3, so 5e-6; the phi
gradient also carries the forward recompute's contraction (about 1e-6, 4e-6 for BF16x3), so 1e-5 and 3e-5;
plain TF32 (10-bit operands in the forward recompute) 5e-5 and 2e-3."""
import numpy as np
import pytest
import torch

import oracle.adjoint as OA
import oracle.healpix as hp
from gpu_util import rel_rms, sky, to_dev

pytestmark = pytest.mark.gpu

api = pytest.importorskip("paper_1307_0719_gb300.api")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _grads(rng, nside, dtype, pol):
    n = hp.npix(nside)
    g = {f: rng.normal(size=n) for f in ("TQU" if pol else "T")}
    gd = {f: torch.from_numpy(v).to("cuda:0", dtype) for f, v in g.items()}
    return g, gd


def _gpu_adjoint(nside, lmax, order, s, gd, precision, pol=True, rotate=True, phi=True):
    plan = api.Plan(nside, lmax, order, pol=pol, precision=precision, rotate=rotate)
    d = to_dev(s)
    out = plan.lens_adjoint(d["T"], d.get("E") if pol else None, d.get("B") if pol else None,
                            d["phi"] if phi else None, gd["T"], gd.get("Q"), gd.get("U"), galpha=True)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    plan.close()
    return res


def _cmp(a, b):
    return rel_rms(np.concatenate([a.real, a.imag]), np.concatenate([b.real, b.imag]))


@pytest.mark.parametrize("nside,lmax,order", [(8, 16, 2), (16, 40, 4), (4, 12, 6), (16, 32, 0), (32, 80, 3)])
def test_adjoint_tqu_fp64(nside, lmax, order):
    s = sky(nside, lmax, pol=True, b_scale=0.5)
    rng = np.random.default_rng(nside + order)
    g, gd = _grads(rng, nside, torch.float64, True)
    ref = OA.lens_adjoint(nside, lmax, order, s["T"], s["E"], s["B"], s["phi"], g["T"], g["Q"], g["U"])
    out = _gpu_adjoint(nside, lmax, order, s, gd, api.FP64)
    for f in "TEB":
        assert _cmp(out[f], ref[f]) < 1e-10, (f, _cmp(out[f], ref[f]))
    assert _cmp(out["phi"], ref["phi"]) < 1e-8, _cmp(out["phi"], ref["phi"])
    for i in range(2):
        # at order 0 the alpha gradient is dL/dbeta dbeta/dalpha alone, and the small
        # d(beta)/d(a_theta) carries the oracle's difference error (~1e-7 relative)
        tol = 5e-7 if (order == 0 and i == 0) else 1e-8
        assert rel_rms(out["alpha"][i], ref["alpha"][i]) < tol, (i, rel_rms(out["alpha"][i], ref["alpha"][i]))
    # m = 0 coefficients are real: no imaginary gradient
    m0 = slice(0, lmax + 1)
    for f in ("T", "E", "B", "phi"):
        assert np.all(out[f][m0].imag == 0.0)


def test_adjoint_t_only_and_unrotated_fp64():
    nside, lmax, order = 16, 40, 3
    s = sky(nside, lmax, pol=True, b_scale=0.5)
    rng = np.random.default_rng(11)
    g, gd = _grads(rng, nside, torch.float64, True)
    # temperature-only plan
    ref = OA.lens_adjoint(nside, lmax, order, s["T"], None, None, s["phi"], g["T"])
    out = _gpu_adjoint(nside, lmax, order, s, gd, api.FP64, pol=False)
    assert _cmp(out["T"], ref["T"]) < 1e-10
    assert _cmp(out["phi"], ref["phi"]) < 1e-8
    assert "E" not in out
    # polarised plan without the rotation R
    ref = OA.lens_adjoint(nside, lmax, order, s["T"], s["E"], s["B"], s["phi"], g["T"], g["Q"], g["U"],
                          rotate=False)
    out = _gpu_adjoint(nside, lmax, order, s, gd, api.FP64, rotate=False)
    for f in ("T", "E", "B"):
        assert _cmp(out[f], ref[f]) < 1e-10, f
    assert _cmp(out["phi"], ref["phi"]) < 1e-8


def test_adjoint_zero_deflection_fp64():
    """alm_phi NULL: alpha = 0 everywhere; the phi gradient is the derivative at phi = 0."""
    nside, lmax, order = 8, 20, 3
    s = sky(nside, lmax, pol=True, b_scale=0.5)
    zero = np.zeros_like(s["phi"])
    rng = np.random.default_rng(5)
    g, gd = _grads(rng, nside, torch.float64, True)
    ref = OA.lens_adjoint(nside, lmax, order, s["T"], s["E"], s["B"], zero, g["T"], g["Q"], g["U"])
    plan = api.Plan(nside, lmax, order, pol=True, precision=api.FP64)
    d = to_dev(s)
    out = plan.lens_adjoint(d["T"], d["E"], d["B"], None, gd["T"], gd["Q"], gd["U"])
    torch.cuda.synchronize()
    for f in ("T", "E", "B"):
        assert _cmp(out[f].cpu().numpy(), ref[f]) < 1e-10, f
    assert _cmp(out["phi"].cpu().numpy(), ref["phi"]) < 1e-8
    plan.close()


def test_adjoint_dot_product_fp64():
    """<y, lens(x)> = Re <lens^T y, x> for (T, E, B) at fixed phi, on the GPU alone."""
    nside, lmax, order = 64, 128, 4
    s = sky(nside, lmax, pol=True, b_scale=0.5)
    rng = np.random.default_rng(2)
    g, gd = _grads(rng, nside, torch.float64, True)
    plan = api.Plan(nside, lmax, order, pol=True, precision=api.FP64)
    d = to_dev(s)
    maps = plan.lens(d["T"], d["E"], d["B"], d["phi"])
    lhs = sum(float(torch.dot(maps[i], gd[f])) for i, f in enumerate("TQU"))
    gr = plan.lens_adjoint(d["T"], d["E"], d["B"], d["phi"], gd["T"], gd["Q"], gd["U"])
    rhs = sum(float((gr[f].conj() * d[f]).real.sum()) for f in "TEB")
    torch.cuda.synchronize()
    plan.close()
    assert abs(lhs - rhs) < 1e-11 * abs(lhs), (lhs, rhs)


@pytest.mark.parametrize("precision,tol_teb,tol_phi", [("MIXED_FP32", 5e-6, 1e-5), ("MIXED_TF32x3", 5e-6, 1e-5),
                                                       ("MIXED_BF16x3", 5e-6, 3e-5), ("MIXED_TF32", 5e-5, 2e-3)])
def test_adjoint_mixed(precision, tol_teb, tol_phi):
    nside, lmax, order = 32, 64, 4
    s = sky(nside, lmax, pol=True, b_scale=0.5)
    rng = np.random.default_rng(21)
    g, gd = _grads(rng, nside, torch.float32, True)
    ref = OA.lens_adjoint(nside, lmax, order, s["T"], s["E"], s["B"], s["phi"], g["T"], g["Q"], g["U"])
    out = _gpu_adjoint(nside, lmax, order, s, gd, getattr(api, precision))
    for f in "TEB":
        assert _cmp(out[f], ref[f]) < tol_teb, (f, _cmp(out[f], ref[f]))
    assert _cmp(out["phi"], ref["phi"]) < tol_phi, _cmp(out["phi"], ref["phi"])


def test_lens_function_autograd_fp64():
    nside, lmax, order = 16, 32, 3
    s = sky(nside, lmax, pol=True, b_scale=0.5)
    rng = np.random.default_rng(8)
    g, gd = _grads(rng, nside, torch.float64, True)
    plan = api.Plan(nside, lmax, order, pol=True, precision=api.FP64)
    d = {k: v.clone().requires_grad_(True) for k, v in to_dev(s).items()}
    y = torch.stack([gd["T"], gd["Q"], gd["U"]])
    out = api.LensFunction.apply(plan, d["T"], d["E"], d["B"], d["phi"])
    loss = (out * y).sum()
    loss.backward()
    ref = OA.lens_adjoint(nside, lmax, order, s["T"], s["E"], s["B"], s["phi"], g["T"], g["Q"], g["U"])
    for f, k in (("T", "T"), ("E", "E"), ("B", "B"), ("phi", "phi")):
        tol = 1e-8 if f == "phi" else 1e-10
        assert _cmp(d[k].grad.cpu().numpy(), ref[f]) < tol, f
    torch.cuda.synchronize()
    plan.close()


def test_adjoint_rejects_bad_arguments():
    nside, lmax, order = 4, 8, 2
    plan = api.Plan(nside, lmax, order, pol=False, precision=api.FP64)
    s = to_dev(sky(nside, lmax, pol=False))
    gT = torch.zeros(hp.npix(nside), dtype=torch.float64, device="cuda:0")
    e = torch.zeros(plan.nalm, dtype=torch.complex128, device="cuda:0")
    from paper_1307_0719_gb300 import _lib
    import ctypes
    L = _lib.lib()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    # E output on a temperature-only plan
    st = L.tl_lens_adjoint(plan._h, p(s["T"]), None, None, p(s["phi"]), p(gT), None, None, None,
                           p(torch.view_as_real(e)), None, None, None, None)
    assert st == _lib.TL_ERR_ARG
    # missing upstream gradient
    st = L.tl_lens_adjoint(plan._h, p(s["T"]), None, None, p(s["phi"]), None, None, None, None, None, None,
                           None, None, None)
    assert st == _lib.TL_ERR_ARG
    plan.close()


def test_adjoint_nside1024_central_differences():
    """Differentiation workload (Nside 1024, lmax 2048, order 4, T+Q/U): the FP64
    tl_lens_adjoint gradient of L = sum (s' - s_target)^2 against central differences
    of the FP64 forward on 32 random coefficients (8 each of T, E, B, phi; real or
    imaginary part), step 1e-6 of the entry. The loss difference is formed per pixel,
    sum (s'+ - s'-)(s'+ + s'- - 2 s_target), so that the step is not lost in the
    rounding of a sum of squares of order 1e11. The phi entries move the deflection,
    and a point that crosses a pixel boundary changes its expansion pixel (the map is
    piecewise smooth in phi; the adjoint holds q fixed): with this step a handful of
    the 12.6 M pixels cross, each changing L by far less than the phi gradient times
    the step, hence the 1e-3 relative tolerance for every entry."""
    import skygen
    w = skygen.WORKLOADS["nside1024_lmax2048_n4_TQU"]
    s = skygen.make_sky(w.nside, w.lmax, True, w.seed_t, w.seed_e, w.seed_phi, w.damp_t, w.damp_e)
    t = skygen.make_sky(w.nside, w.lmax, True, 9000, 9001, 9002, w.damp_t, w.damp_e)
    d, dt = to_dev(s), to_dev(t)
    plan = api.Plan(w.nside, w.lmax, w.order, pol=True, precision=api.FP64)
    try:
        target = plan.lens(dt["T"], dt["E"], dt["B"], dt["phi"]).clone()
        out = plan.lens(d["T"], d["E"], d["B"], d["phi"]).clone()
        g = 2.0 * (out - target)
        gr = plan.lens_adjoint(d["T"], d["E"], d["B"], d["phi"], g[0].contiguous(), g[1].contiguous(),
                               g[2].contiguous())
        gr = {k: v.cpu().numpy() for k, v in gr.items()}
        rng = np.random.default_rng(4)
        lmax = w.lmax
        checks = []
        for f, lhi in (("T", 300), ("E", 300), ("B", 300), ("phi", 100)):
            n = 0
            while n < 8:
                l = int(rng.integers(2, lhi))
                m = int(rng.integers(0, l + 1))
                idx = m * (2 * lmax + 1 - m) // 2 + l
                # B = 0 in this workload: its step takes the scale of E at the same (l, m)
                scale = abs(complex(s[f][idx])) if f != "B" else abs(complex(s["E"][idx]))
                if scale == 0.0:
                    continue
                part = "re" if (m == 0 or rng.random() < 0.5) else "im"
                h = 1e-6 * scale
                pm = []
                for sgn in (1.0, -1.0):
                    dd = dict(d)
                    v = dd[f].clone()
                    v[idx] += sgn * h * (1.0 if part == "re" else 1j)
                    dd[f] = v
                    pm.append(plan.lens(dd["T"], dd["E"], dd["B"], dd["phi"]).clone())
                fd = float(((pm[0] - pm[1]) * (pm[0] + pm[1] - 2.0 * target)).sum()) / (2.0 * h)
                ana = gr[f][idx].real if part == "re" else gr[f][idx].imag
                checks.append((f, l, m, part, fd, ana))
                n += 1
    finally:
        torch.cuda.synchronize()
        plan.close()
    for f, l, m, part, fd, ana in checks:
        assert abs(fd - ana) <= 1e-3 * abs(ana), (f, l, m, part, fd, ana)


@pytest.mark.parametrize("nside,lmax,precision", [(1024, 2048, "MIXED_FP32"), (2048, 4096, "MIXED_BF16x3")])
def test_adjoint_dot_product_mixed_full_size(nside, lmax, precision):
    """The transpose identity <y, lens(x)> = Re <lens^T y, x> for (T, E, B) at fixed phi
    at the sizes where the adjoint ring FFT runs its register Bluestein sub-transforms
    (cap rings with 513 <= i <= 2047), in single precision (float sums over 12.6M and
    50M pixels: 1e-4)."""
    s = sky(nside, lmax, pol=True, b_scale=0.5)
    rng = np.random.default_rng(5)
    g, gd = _grads(rng, nside, torch.float32, True)
    plan = api.Plan(nside, lmax, 4, pol=True, precision=getattr(api, precision))
    try:
        d = to_dev(s)
        maps = plan.lens(d["T"], d["E"], d["B"], d["phi"]).double()
        lhs = sum(float(torch.dot(maps[i], gd[f].double())) for i, f in enumerate("TQU"))
        gr = plan.lens_adjoint(d["T"], d["E"], d["B"], d["phi"], gd["T"], gd["Q"], gd["U"], want=("T", "E", "B"))
        rhs = sum(float((gr[f].conj() * d[f]).real.sum()) for f in "TEB")
    finally:
        torch.cuda.synchronize()
        plan.close()
    assert abs(lhs - rhs) < 1e-4 * abs(lhs), (lhs, rhs)
