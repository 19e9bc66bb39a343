"""Pins for the oracle's derivative-map synthesis, displacement, pixel-relative
Taylor sum (Eq. 4) and polarisation rotation (Eq. 2) -- Naess & Louis 2013, Sec. II."""
from math import factorial

import numpy as np
import pytest

import oracle.healpix as hp
import oracle.lens as L
import oracle.sht as sht
import skygen


def _single_mode(lmax, l, m, val):
    a = np.zeros(skygen.alm_size(lmax), dtype=np.complex128)
    a[skygen.alm_index(lmax, l, m)] = val
    return a


def test_zero_displacement_is_identity_bitexact():
    """alpha = 0: x' = x, the expansion pixel is p itself, every offset is 0, and
    the output is exactly the order-0 map (Sec. II.B)."""
    sky = skygen.make_sky(16, 32, True, 0, 3, 1, b_scale=0.3)
    zero = np.zeros_like(sky["phi"])
    out = L.lens(16, 32, 4, sky["T"], sky["E"], sky["B"], zero, return_aux=True)
    base = L.derivative_maps(16, 32, 0, sky["T"], sky["E"], sky["B"])
    for f in "TQU":
        assert np.array_equal(out[f], base[f][0])
    assert np.array_equal(out["aux"]["q"], np.arange(hp.npix(16)))


def test_pure_E_and_B_m0_conventions():
    """Q +- iU = -sum (E +- iB) +-2Y (HEALPix): a pure E_l0 gives U = 0 and a pure
    B_l0 gives Q = 0, because +-2Y_l0 are real and equal."""
    lmax = 12
    E = _single_mode(lmax, 5, 0, 1.0)
    Z = np.zeros_like(E)
    m = L.derivative_maps(8, lmax, 2, alm_E=E, alm_B=Z)
    assert np.abs(m["U"]).max() < 1e-14 and np.abs(m["Q"]).max() > 0.1
    m = L.derivative_maps(8, lmax, 2, alm_E=Z, alm_B=E)
    assert np.abs(m["Q"]).max() < 1e-14 and np.abs(m["U"]).max() > 0.1


def test_single_mode_derivatives_closed_form():
    """T = 2 Re[a Y_32]: every d_theta^j d_phi^k map equals the symbolic derivative
    of the textbook Y_32 at the pixel centres."""
    sp = pytest.importorskip("sympy")
    th, ph = sp.symbols("theta phi", real=True)
    a = 0.7 - 0.4j
    Y = sp.Ynm(3, 2, th, ph).expand(func=True)
    T = 2 * sp.re(sp.expand((sp.Float(a.real) + sp.I * sp.Float(a.imag)) * Y, complex=True))
    nside, lmax, n = 8, 6, 3
    maps = L.derivative_maps(nside, lmax, n, alm_T=_single_mode(lmax, 3, 2, a))["T"]
    thp, php = hp.pix2ang(nside, np.arange(hp.npix(nside)))
    for (j, k) in L.derivative_pairs(n):
        f = sp.lambdify((th, ph), sp.diff(T, th, j, ph, k), "numpy")
        ref = np.broadcast_to(f(thp, php), thp.shape)
        assert np.allclose(maps[L.map_index(j, k)], ref, atol=1e-12), (j, k)


def test_spin2_single_mode_closed_form():
    """Q + iU = -(E_21 2Y_21 + E_2,-1 2Y_2,-1) with E_2,-1 = -conj(E_21) and the
    textbook 2Y_2m of Goldberg et al. (1967), from their explicit sum formula:
    2Y_21 = -sqrt(5/(16 pi)) sin(th)(1 - cos th) e^{i phi},
    2Y_2,-1 = -sqrt(5/(16 pi)) sin(th)(1 + cos th) e^{-i phi}."""
    lmax = 4
    e = 0.3 + 0.8j
    maps = L.derivative_maps(4, lmax, 0, alm_E=_single_mode(lmax, 2, 1, e),
                             alm_B=np.zeros(skygen.alm_size(lmax), complex))
    th, ph = hp.pix2ang(4, np.arange(hp.npix(4)))
    c = np.sqrt(5 / (16 * np.pi))
    y21 = -c * np.sin(th) * (1 - np.cos(th)) * np.exp(1j * ph)
    y2m1 = -c * np.sin(th) * (1 + np.cos(th)) * np.exp(-1j * ph)
    P = -(e * y21 + (-np.conj(e)) * y2m1)
    assert np.allclose(maps["Q"][0], P.real, atol=1e-13)
    assert np.allclose(maps["U"][0], P.imag, atol=1e-13)


def test_fft_ring_synthesis_equals_direct_sum():
    sky = skygen.make_sky(32, 64, True, 5, 6, 7, b_scale=0.5)
    maps = L.derivative_maps(32, 64, 3, sky["T"], sky["E"], sky["B"])
    pix = np.random.default_rng(1).choice(hp.npix(32), 300, replace=False)
    th, ph = hp.pix2ang(32, pix)
    F = sht.ring_coeffs(64, 3, th, sky["T"], sky["E"], sky["B"])
    for f in "TQU":
        for (j, k) in L.derivative_pairs(3):
            d = sht.point_sum(F[f], ph, j, k)
            ref = maps[f][L.map_index(j, k), pix]
            assert np.allclose(d, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("nside,lmax", [(32, 32), (64, 64)])
def test_converges_to_brute_force(nside, lmax):
    """Error against direct spherical-harmonic sums at the displaced points
    (the exact Born remap, Eqs. 1-2) falls with the order and reaches rounding."""
    sky = skygen.make_sky(nside, lmax, True, 0, 3, 1, b_scale=0.5)
    pix = np.random.default_rng(0).choice(hp.npix(nside), 600, replace=False)
    ex = L.lens_exact(nside, lmax, sky["T"], sky["E"], sky["B"], sky["phi"], pix=pix)
    errs = []
    for n in range(0, 10):
        o = L.lens_at_pixels(nside, lmax, n, pix, sky["T"], sky["E"], sky["B"], sky["phi"])
        errs.append(max(np.sqrt(np.mean((o[f] - ex[f]) ** 2) / np.mean(ex[f] ** 2)) for f in "TQU"))
    errs = np.array(errs)
    assert np.all(np.diff(errs[:6]) < 0), errs
    assert errs[1] < 0.05 * errs[0] and errs[3] < 1e-5
    assert errs[9] < 1e-12, errs


def test_order_n_matches_truncated_series_closed_form():
    """Single mode T = 2 Re[a Y_lm], given offsets: Eq. 4 equals the hand-built
    truncated series sum dth^j dph^k/(j!k!) d^j lambda (i m)^k e^{i m phi} (with the
    derivative of lambda from exact Fourier differentiation, not the oracle's ladder)."""
    l, m, a = 9, 4, 0.3 + 1.1j
    lmax, nside, n = 12, 16, 5
    maps = L.derivative_maps(nside, lmax, n, alm_T=_single_mode(lmax, l, m, a))["T"]
    rng = np.random.default_rng(2)
    q = rng.choice(hp.npix(nside), 50, replace=False)
    dth = rng.uniform(-0.03, 0.03, 50)
    dph = rng.uniform(-0.03, 0.03, 50)
    got = L.taylor_sum(maps[:, q], dth, dph, n)
    thq, phq = hp.pix2ang(nside, q)
    N = 2 * l + 2
    grid = (np.arange(N) + 0.5) * 2 * np.pi / N
    vals = np.array([sht.spin_lambda(l, m, 0, t)[l] for t in grid])
    kk = np.fft.fftfreq(N, 1.0 / N)
    c = np.fft.fft(vals) / N * np.exp(-1j * kk * np.pi / N)
    ref = np.zeros(50)
    for j in range(n + 1):
        for k in range(n + 1 - j):
            dl = np.array([np.sum(c * (1j * kk) ** j * np.exp(1j * kk * t)).real for t in thq])
            term = 2 * (a * dl * (1j * m) ** k * np.exp(1j * m * phq)).real
            ref += dth ** j * dph ** k / (factorial(j) * factorial(k)) * term
    assert np.allclose(got, ref, atol=1e-11 * np.abs(ref).max())


def test_pure_phi_offset_is_truncated_exponential():
    """With dth = 0 the sum over k of (i m dph)^k/k! multiplies each m-mode: check
    against exp(i m dph) truncated, for a single mode."""
    l, m, a, lmax, nside, n = 6, 5, 1.0 + 0.0j, 8, 8, 6
    maps = L.derivative_maps(nside, lmax, n, alm_T=_single_mode(lmax, l, m, a))["T"]
    q = np.arange(hp.npix(nside))
    dph = np.full(q.size, 0.05)
    got = L.taylor_sum(maps[:, q], np.zeros(q.size), dph, n)
    base = maps[L.map_index(0, 0)]
    # T = 2 Re[w], w = a lam e^{i m phi}; dT/dphi = -2 m Im[w]
    quad = -maps[L.map_index(0, 1)] / m  # = 2 Im[w]
    z = base + 1j * quad  # = 2 w
    trunc = sum((1j * m * 0.05) ** k / factorial(k) for k in range(n + 1))
    assert np.allclose(got, (z * trunc).real, atol=1e-13)


def test_rotation_3d_tensor():
    """Polarisation of a constant 3D symmetric tensor M, P(y) = m(y)^T M m(y) with
    m = e_theta + i e_phi (a spin-2 field). Carried from x' back to x by parallel
    transport along the geodesic (a 3D rotation about n x u by -d), it must equal
    exp(-2 i beta) P(x') with the oracle's beta."""
    rng = np.random.default_rng(11)
    A = rng.normal(size=(3, 3))
    M = A + A.T
    K = 2000
    z = rng.uniform(-0.999, 0.999, K)
    s = np.sqrt(1 - z * z)
    phi = rng.uniform(0, 2 * np.pi, K)
    a_th = rng.normal(0, 0.05, K)
    a_ph = rng.normal(0, 0.05, K)
    n2, u, n, et, d = L.displace(z, s, phi, a_th, a_ph)
    th2 = np.arctan2(np.hypot(n2[:, 0], n2[:, 1]), n2[:, 2])
    ph2 = np.arctan2(n2[:, 1], n2[:, 0])
    beta = L.transport_angle(n, u, et, d, th2, ph2)
    _, et2, ep2 = L.basis(th2, ph2)
    m2 = et2 + 1j * ep2
    P2 = np.einsum("ki,ij,kj->k", m2, M, m2)
    # transport: the rotation R taking n to n2 maps m(x) to a tangent frame at x';
    # the transported tensor read at x is (R m)^T M (R m)
    _, et1, ep1 = L.basis_zs(z, s, phi)
    axis = np.cross(n, u)
    Rm = L.rotate_about(et1, axis, d) + 1j * L.rotate_about(ep1, axis, d)
    Ptrans = np.einsum("ki,ij,kj->k", Rm, M, Rm)
    assert np.allclose(Ptrans, np.exp(-2j * beta) * P2, atol=1e-12)
    # beta -> 0 as d -> 0
    n2, u, n, et, d = L.displace(z, s, phi, a_th * 1e-9, a_ph * 1e-9)
    th2 = np.arctan2(np.hypot(n2[:, 0], n2[:, 1]), n2[:, 2])
    ph2 = np.arctan2(n2[:, 1], n2[:, 0])
    assert np.abs(L.transport_angle(n, u, et, d, th2, ph2)).max() < 1e-6


def test_geodesic_invariants_and_naive_limit():
    rng = np.random.default_rng(4)
    K = 5000
    z = rng.uniform(-0.99, 0.99, K)
    s = np.sqrt(1 - z * z)
    phi = rng.uniform(0, 2 * np.pi, K)
    a_th = rng.normal(0, 1e-3, K)
    a_ph = rng.normal(0, 1e-3, K)
    n2, u, n, et, d = L.displace(z, s, phi, a_th, a_ph)
    assert np.allclose(np.linalg.norm(n2, axis=1), 1, atol=1e-15)
    ang = np.arctan2(np.linalg.norm(np.cross(n, n2), axis=1), np.sum(n * n2, axis=1))
    assert np.allclose(ang, d, rtol=1e-9)
    th = np.arccos(z)
    th2 = np.arctan2(np.hypot(n2[:, 0], n2[:, 1]), n2[:, 2])
    ph2 = np.arctan2(n2[:, 1], n2[:, 0])
    # naive coordinate addition agrees to second order in |alpha|
    assert np.abs(th2 - (th + a_th)).max() < 50 * d.max() ** 2 / s.min()
    dphi = L.wrap_pi(ph2 - phi - a_ph / s)
    assert np.abs(dphi * s).max() < 50 * d.max() ** 2 / s.min()


def test_linearity_in_unlensed_fields():
    sky1 = skygen.make_sky(16, 32, True, 0, 3, 1, b_scale=0.2)
    sky2 = skygen.make_sky(16, 32, True, 8, 9, 1, b_scale=0.7)
    a, b = 1.7, -0.6
    o1 = L.lens(16, 32, 3, sky1["T"], sky1["E"], sky1["B"], sky1["phi"])
    o2 = L.lens(16, 32, 3, sky2["T"], sky2["E"], sky2["B"], sky1["phi"])
    o = L.lens(16, 32, 3, a * sky1["T"] + b * sky2["T"], a * sky1["E"] + b * sky2["E"],
               a * sky1["B"] + b * sky2["B"], sky1["phi"])
    for f in "TQU":
        assert np.allclose(o[f], a * o1[f] + b * o2[f], atol=1e-12 * np.abs(o[f]).max())


def test_deflection_quantile_matches_paper():
    """The paper's simulations have a 99% quantile of the deflection of 5.3 arcmin
    (Fig. 1 caption); a 2.5' RMS Gaussian deflection gives 5.37' (Rayleigh)."""
    sky = skygen.make_sky(256, 512, False, 0, 0, 1)
    a_th, a_ph = L.deflection(256, 512, sky["phi"])
    q99 = np.quantile(np.hypot(a_th, a_ph), 0.99) / skygen.ARCMIN
    assert 4.8 < q99 < 5.9, q99


def test_deflection_closed_forms_Y10_Y11():
    """alpha = (d_theta phi, d_phi phi / sin theta) (Sec. I) for phi = Y_10 and
    phi = 2 Re[a Y_11]: with Y_10 = sqrt(3/4pi) cos th and Y_11 = -sqrt(3/8pi) sin th
    e^{i ph}, alpha_theta = -sqrt(3/4pi) sin th, alpha_phi = 0, and for a = ar + i ai
    alpha_theta = -sqrt(3/2pi) cos th (ar cos ph - ai sin ph),
    alpha_phi = sqrt(3/2pi) (ar sin ph + ai cos ph): smooth, so a dropped or doubled
    1/sin theta shows at every ring."""
    nside, lmax = 8, 4
    th, ph = hp.pix2ang(nside, np.arange(hp.npix(nside)))
    a_th, a_ph = L.deflection(nside, lmax, _single_mode(lmax, 1, 0, 1.0))
    assert np.allclose(a_th, -np.sqrt(3 / (4 * np.pi)) * np.sin(th), atol=1e-13, rtol=0)
    assert np.abs(a_ph).max() < 1e-13
    ar, ai = 0.8, -0.35
    a_th, a_ph = L.deflection(nside, lmax, _single_mode(lmax, 1, 1, ar + 1j * ai))
    c = np.sqrt(3 / (2 * np.pi))
    assert np.allclose(a_th, -c * np.cos(th) * (ar * np.cos(ph) - ai * np.sin(ph)), atol=1e-13, rtol=0)
    assert np.allclose(a_ph, c * (ar * np.sin(ph) + ai * np.cos(ph)), atol=1e-13, rtol=0)


@pytest.mark.parametrize("order", [0, 1, 2, 3, 4, 5, 6])
def test_lens_equals_sampled_evaluator(order):
    """The whole-map oracle (derivative maps by ring FFTs, deflection maps, the
    gather at q of every pixel) against the sampled evaluator, which takes every
    step by direct sums at the points themselves (the deflection on the pixel's
    ring, the derivative values at q from direct Fourier sums); the latter is pinned
    to brute-force Y_lm sums by test_convergence_to_brute_force. phi is scaled up so
    that the deflections move most points out of their own pixel."""
    nside, lmax = 16, 40
    sky = skygen.make_sky(nside, lmax, True, 0, 3, 1, b_scale=0.4)
    phi = sky["phi"] * 200.0
    full = L.lens(nside, lmax, order, sky["T"], sky["E"], sky["B"], phi, return_aux=True)
    moved = np.mean(full["aux"]["q"] != np.arange(hp.npix(nside)))
    assert moved > 0.5, moved
    pix = np.arange(hp.npix(nside))
    samp = L.lens_at_pixels(nside, lmax, order, pix, sky["T"], sky["E"], sky["B"], phi)
    assert np.array_equal(samp["aux"]["q"], full["aux"]["q"])
    for f in "TQU":
        scale = np.sqrt(np.mean(full[f] ** 2))
        assert np.abs(samp[f] - full[f]).max() < 1e-12 * scale, (f, np.abs(samp[f] - full[f]).max() / scale)


def test_naive_displacement_meridian_equals_geodesic_across_pole():
    """Naive coordinate addition (Sec. II.A's alternative) for a deflection along
    e_theta only: the geodesic is then the meridian, so both give the same x',
    including points carried past a pole (theta' = -theta, phi' = phi + pi)."""
    rng = np.random.default_rng(7)
    K = 2000
    th = rng.uniform(1e-3, np.pi - 1e-3, K)
    phi = rng.uniform(0, 2 * np.pi, K)
    a_th = rng.uniform(-0.5, 0.5, K)
    a_th[:200] = -th[:200] - rng.uniform(1e-3, 0.2, 200)        # past the north pole
    a_th[200:400] = np.pi - th[200:400] + rng.uniform(1e-3, 0.2, 200)  # past the south pole
    z, s = np.cos(th), np.sin(th)
    zero = np.zeros(K)
    tn, pn, zn, sn, _ = L.target_point(th, z, s, phi, a_th, zero, naive=True)
    tg, pg, zg, sg, _ = L.target_point(th, z, s, phi, a_th, zero, naive=False)
    assert np.allclose(tn, tg, atol=1e-12)
    assert np.allclose(np.abs(L.wrap_pi(pn - pg)) * sg, 0.0, atol=1e-12)


def test_naive_displacement_second_order_agreement():
    """For small deflections naive addition and the geodesic end point differ at
    second order in |alpha| (transverse to the meridian), so the lensed maps do too."""
    nside, lmax, n = 16, 32, 4
    sky = skygen.make_sky(nside, lmax, True, 0, 3, 1, b_scale=0.4)
    diffs = []
    for scale in (10.0, 20.0):
        phi = sky["phi"] * scale
        g = L.lens(nside, lmax, n, sky["T"], sky["E"], sky["B"], phi, return_aux=True)
        nv = L.lens(nside, lmax, n, sky["T"], sky["E"], sky["B"], phi, naive=True)
        diffs.append(max(np.sqrt(np.mean((nv[f] - g[f]) ** 2) / np.mean(g[f] ** 2)) for f in "TQU"))
    # doubling the deflection multiplies the difference by about four (second order)
    assert 2.5 < diffs[1] / diffs[0] < 6.0, diffs


def test_expansion_about_the_pixel_itself():
    """The plain Taylor series about the undisplaced point (Sec. I, Eq. 3a; q = p):
    zero deflection returns the order-0 map exactly; with deflections the error
    against brute-force Y_lm sums falls with the order; and at a fixed low order it is
    larger than the pixel-relative expansion about the cell containing x' (the
    paper's motivation, Fig. 1), for deflections of several pixels."""
    nside, lmax = 32, 32
    sky = skygen.make_sky(nside, lmax, True, 0, 3, 1, b_scale=0.5)
    zero = np.zeros_like(sky["phi"])
    o = L.lens(nside, lmax, 4, sky["T"], sky["E"], sky["B"], zero, at_pixel=True)
    base = L.derivative_maps(nside, lmax, 0, sky["T"], sky["E"], sky["B"])
    for f in "TQU":
        assert np.array_equal(o[f], base[f][0])
    phi = sky["phi"] * 30.0
    pix = np.random.default_rng(3).choice(hp.npix(nside), 400, replace=False)
    ex = L.lens_exact(nside, lmax, sky["T"], sky["E"], sky["B"], phi, pix=pix)

    def err(n, at_pixel):
        r = L.lens_at_pixels(nside, lmax, n, pix, sky["T"], sky["E"], sky["B"], phi, at_pixel=at_pixel)
        return max(np.sqrt(np.mean((r[f] - ex[f]) ** 2) / np.mean(ex[f] ** 2)) for f in "TQU")
    e_px = [err(n, True) for n in (1, 3, 5, 8, 12)]
    assert np.all(np.diff(e_px) < 0) and e_px[-1] < 1e-6, e_px
    assert err(2, True) > 2.0 * err(2, False)


def test_map2alm_is_the_weighted_transpose_of_synthesis():
    """map2alm (uniform weights w = 4 pi / Npix) against the synthesis of the
    derivative-map code (an independent route, one FFT per ring): for real fields,
    sum_lm c_m Re(a_lm conj(map2alm(m)_lm)) = w sum_p m(p) synth(a)(p), c_0 = 1,
    c_m>0 = 2, for T and for (E, B) <-> (Q, U), to rounding."""
    nside, lmax = 16, 24
    w = 4 * np.pi / hp.npix(nside)
    a = skygen.make_sky(nside, lmax, True, 0, 3, 1, b_scale=0.6)
    syn = L.derivative_maps(nside, lmax, 0, a["T"], a["E"], a["B"])
    rng = np.random.default_rng(0)
    mT, mQ, mU = (rng.normal(size=hp.npix(nside)) for _ in range(3))
    b = L.map2alm(nside, lmax, mT, mQ, mU)
    c = np.full(skygen.alm_size(lmax), 2.0)
    c[:lmax + 1] = 1.0
    lhs = np.sum(c * (a["T"] * np.conj(b["T"])).real)
    rhs = w * np.sum(mT * syn["T"][0])
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    lhs = np.sum(c * ((a["E"] * np.conj(b["E"])).real + (a["B"] * np.conj(b["B"])).real))
    rhs = w * np.sum(mQ * syn["Q"][0] + mU * syn["U"][0])
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_map2alm_recovers_band_limited_coefficients():
    """Analysis after synthesis returns the coefficients up to the quadrature error of
    the HEALPix grid with uniform weights (about 1e-3 at lmax = 2 nside)."""
    nside, lmax = 32, 64
    a = skygen.make_sky(nside, lmax, True, 0, 3, 1, b_scale=0.5)
    m = L.derivative_maps(nside, lmax, 0, a["T"], a["E"], a["B"])
    b = L.map2alm(nside, lmax, m["T"][0], m["Q"][0], m["U"][0])
    for f in "TEB":
        err = np.sqrt(np.sum(np.abs(b[f] - a[f]) ** 2) / np.sum(np.abs(a[f]) ** 2))
        assert err < 1e-2, (f, err)


def test_anafast_single_modes():
    """C_l of one coefficient: |a|^2 / (2l+1) for m = 0 and 2 |a|^2 / (2l+1) for m > 0
    (a_l,-m carries the same power); cross spectra take Re(x conj(y))."""
    lmax = 10
    x = _single_mode(lmax, 4, 0, 1.5)
    assert np.allclose(L.anafast(lmax, x), np.where(np.arange(lmax + 1) == 4, 2.25 / 9, 0.0))
    x = _single_mode(lmax, 6, 3, 0.6 - 0.8j)
    y = _single_mode(lmax, 6, 3, 2.0j)
    assert np.allclose(L.anafast(lmax, x), np.where(np.arange(lmax + 1) == 6, 2 * 1.0 / 13, 0.0))
    assert np.allclose(L.anafast(lmax, x, y), np.where(np.arange(lmax + 1) == 6, 2 * (-1.6) / 13, 0.0))


def test_lmax_phi_default_is_the_plan_lmax_and_matches_brute_force():
    """The potential's own band limit (Sec. II.A: the gradient map is taken to
    min(8 Nside, 10000)): lmax_phi = lmax is the default exactly, and with a larger
    lmax_phi the lensed maps converge with order to the brute-force remap whose
    deflection comes from direct sums at the same lmax_phi (an independent route:
    point sums instead of ring FFTs)."""
    nside, lmax = 16, 24
    sky = skygen.make_sky(nside, lmax, True, 0, 3, 1, b_scale=0.4)
    a = L.lens(nside, lmax, 3, sky["T"], sky["E"], sky["B"], sky["phi"])
    b = L.lens(nside, lmax, 3, sky["T"], sky["E"], sky["B"], sky["phi"], lmax_phi=lmax)
    for f in "TQU":
        assert np.array_equal(a[f], b[f])
    lp = 8 * nside
    phi = skygen.make_sky(nside, lp, False, 0, 0, 5)["phi"] * 5.0
    pix = np.random.default_rng(2).choice(hp.npix(nside), 300, replace=False)
    ex = L.lens_exact(nside, lmax, sky["T"], sky["E"], sky["B"], phi, pix=pix, lmax_phi=lp)
    errs = []
    for n in (1, 3, 6):
        r = L.lens_at_pixels(nside, lmax, n, pix, sky["T"], sky["E"], sky["B"], phi, lmax_phi=lp)
        errs.append(max(np.sqrt(np.mean((r[f] - ex[f]) ** 2) / np.mean(ex[f] ** 2)) for f in "TQU"))
    assert np.all(np.diff(errs) < 0) and errs[-1] < 1e-6, errs
    # the modes above lmax move the maps: truncating the potential to lmax changes them
    t = L.lens_at_pixels(nside, lmax, 6, pix, sky["T"], sky["E"], sky["B"], phi[:skygen.alm_size(lmax)] * 0.0,
                         lmax_phi=lmax)
    high = phi.copy()
    high[:] = 0.0
    ells = np.concatenate([np.arange(m, lp + 1) for m in range(lp + 1)])
    high[ells > lmax] = phi[ells > lmax]
    h = L.lens_at_pixels(nside, lmax, 6, pix, sky["T"], sky["E"], sky["B"], high, lmax_phi=lp)
    assert max(np.sqrt(np.mean((h[f] - t[f]) ** 2) / np.mean(t[f] ** 2)) for f in "TQU") > 1e-4
