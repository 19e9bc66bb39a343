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
