"""Pins for the oracle's adjoint (transpose) of Taylor lensing."""
import numpy as np
import pytest

import oracle.adjoint as A
import oracle.healpix as hp
import oracle.lens as L
import skygen


def _dot_alm(a, b):
    return float(np.sum(a.real * b.real + a.imag * b.imag))


def test_dot_product_fixed_deflection():
    """<y, lens(x)> = <lens^T y, x> for the unlensed fields (linear for fixed phi)."""
    nside, lmax, order = 16, 32, 4
    sky = skygen.make_sky(nside, lmax, True, 1, 2, 3, b_scale=0.6)
    rng = np.random.default_rng(9)
    y = {f: rng.normal(size=hp.npix(nside)) for f in "TQU"}
    out = L.lens(nside, lmax, order, sky["T"], sky["E"], sky["B"], sky["phi"])
    lhs = sum(np.dot(y[f], out[f]) for f in "TQU")
    gr = A.lens_adjoint(nside, lmax, order, sky["T"], sky["E"], sky["B"], sky["phi"], y["T"], y["Q"], y["U"])
    rhs = _dot_alm(gr["T"], sky["T"]) + _dot_alm(gr["E"], sky["E"]) + _dot_alm(gr["B"], sky["B"])
    assert abs(lhs - rhs) < 1e-11 * abs(lhs), (lhs, rhs)


def test_phi_gradient_matches_central_differences():
    """dL/dphi_lm against central differences of the full forward map, for
    L = sum_p y . s'(p), at a few coefficients (real and imaginary parts)."""
    nside, lmax, order = 16, 32, 3
    sky = skygen.make_sky(nside, lmax, True, 4, 5, 6, b_scale=0.4)
    rng = np.random.default_rng(3)
    y = {f: rng.normal(size=hp.npix(nside)) for f in "TQU"}

    def loss(phi):
        o = L.lens(nside, lmax, order, sky["T"], sky["E"], sky["B"], phi)
        return sum(np.dot(y[f], o[f]) for f in "TQU")

    gr = A.lens_adjoint(nside, lmax, order, sky["T"], sky["E"], sky["B"], sky["phi"], y["T"], y["Q"], y["U"])
    for (l, m, part) in [(2, 0, 0), (5, 3, 0), (5, 3, 1), (11, 7, 1), (20, 1, 0)]:
        idx = skygen.alm_index(lmax, l, m)
        h = 1e-4 * np.abs(sky["phi"][idx]) + 1e-12
        e = np.zeros_like(sky["phi"])
        e[idx] = h if part == 0 else 1j * h
        fd = (loss(sky["phi"] + e) - loss(sky["phi"] - e)) / (2 * h)
        an = gr["phi"][idx].real if part == 0 else gr["phi"][idx].imag
        assert abs(fd - an) <= 1e-5 * max(abs(fd), abs(an)) + 1e-6 * np.abs(gr["phi"]).max(), (l, m, part, fd, an)


def test_unlensed_gradient_matches_central_differences():
    nside, lmax, order = 8, 16, 2
    sky = skygen.make_sky(nside, lmax, True, 7, 8, 9, b_scale=0.5)
    rng = np.random.default_rng(4)
    y = {f: rng.normal(size=hp.npix(nside)) for f in "TQU"}
    gr = A.lens_adjoint(nside, lmax, order, sky["T"], sky["E"], sky["B"], sky["phi"], y["T"], y["Q"], y["U"])

    def loss(T, E, B):
        o = L.lens(nside, lmax, order, T, E, B, sky["phi"])
        return sum(np.dot(y[f], o[f]) for f in "TQU")

    for field, (l, m) in [("T", (3, 2)), ("E", (4, 1)), ("B", (6, 4)), ("E", (2, 0))]:
        idx = skygen.alm_index(lmax, l, m)
        for part in (0, 1):
            if m == 0 and part == 1:
                continue
            args = {k: sky[k].copy() for k in "TEB"}
            h = 1e-3
            args[field][idx] += h if part == 0 else 1j * h
            lp = loss(args["T"], args["E"], args["B"])
            args[field][idx] -= 2 * (h if part == 0 else 1j * h)
            lm = loss(args["T"], args["E"], args["B"])
            fd = (lp - lm) / (2 * h)
            an = gr[field][idx].real if part == 0 else gr[field][idx].imag
            assert abs(fd - an) < 1e-8 * max(1.0, abs(fd)), (field, l, m, part, fd, an)


def test_geometry_jacobian_accuracy():
    """The Richardson Jacobian of (theta', phi', beta) against 40-digit central
    differences of the same construction (displacement along the geodesic,
    Rodrigues rotation of e_theta about n x u), at points from the pole to the
    equator; error measured against the largest entry of each row."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40

    def geo(z, s, phi, ath, aph):
        z, s, phi, ath, aph = (mp.mpf(v) for v in (z, s, phi, ath, aph))
        cp, sp = mp.cos(phi), mp.sin(phi)
        n = [s * cp, s * sp, z]
        et = [z * cp, z * sp, -s]
        ep = [-sp, cp, mp.mpf(0)]
        d = mp.sqrt(ath ** 2 + aph ** 2)
        u = [(ath * a + aph * b) / d for a, b in zip(et, ep)]
        n2 = [mp.cos(d) * a + mp.sin(d) * b for a, b in zip(n, u)]
        ax = [n[1] * u[2] - n[2] * u[1], n[2] * u[0] - n[0] * u[2], n[0] * u[1] - n[1] * u[0]]
        cr = [ax[1] * et[2] - ax[2] * et[1], ax[2] * et[0] - ax[0] * et[2], ax[0] * et[1] - ax[1] * et[0]]
        dot = sum(a * b for a, b in zip(ax, et))
        t = [a * mp.cos(d) + b * mp.sin(d) + c * dot * (1 - mp.cos(d)) for a, b, c in zip(et, cr, ax)]
        th2 = mp.atan2(mp.sqrt(n2[0] ** 2 + n2[1] ** 2), n2[2])
        ph2 = mp.atan2(n2[1], n2[0])
        et2 = [mp.cos(th2) * mp.cos(ph2), mp.cos(th2) * mp.sin(ph2), -mp.sin(th2)]
        ep2 = [-mp.sin(ph2), mp.cos(ph2), mp.mpf(0)]
        beta = mp.atan2(sum(a * b for a, b in zip(t, ep2)), sum(a * b for a, b in zip(t, et2)))
        return th2, ph2, beta

    rng = np.random.default_rng(3)
    hh = mp.mpf("1e-15")
    for th, sc in [(0.042, 1e-3), (0.1, 7e-4), (1.0, 7e-4), (3.1, 7e-4), (0.02, 5e-3)]:
        for _ in range(3):
            phi = rng.uniform(0, 2 * np.pi)
            ath, aph = rng.normal(scale=sc, size=2)
            z, s = np.cos(th), np.sin(th)
            J = A._jacobian(np.array([z]), np.array([s]), np.array([phi]), np.array([ath]), np.array([aph]),
                            np.array([0.0]), np.array([0.0]))
            for comp, (e0, e1) in enumerate(((1, 0), (0, 1))):
                fp = geo(z, s, phi, ath + hh * e0, aph + hh * e1)
                fm = geo(z, s, phi, ath - hh * e0, aph - hh * e1)
                ref = [float((a - b) / (2 * hh)) for a, b in zip(fp, fm)]
                scale = max(abs(v) for v in ref)
                for q in range(3):
                    assert abs(J[comp][q][0] - ref[q]) < 1e-9 * scale, (th, comp, q, J[comp][q][0], ref[q])
