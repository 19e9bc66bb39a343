"""Pins for the oracle's spin-weighted harmonics and their theta derivatives
(the derivatives of Eq. 4 of the paper, Sec. II.B)."""
from math import factorial, pi, sqrt

import numpy as np
import pytest

import oracle.sht as sht


def test_spin0_matches_scipy():
    from scipy.special import sph_harm_y
    for th in (0.013, 0.4, 1.3, 2.2, 3.1):
        for m in (0, 1, 5, 17, 40):
            lam = sht.spin_lambda(50, m, 0, th)
            for l in range(m, 51):
                ref = sph_harm_y(l, m, th, 0.0).real
                assert abs(lam[l] - ref) <= 1e-12 * max(1.0, abs(ref)), (th, l, m)


def _sympy_spin_Y(l, m, s):
    """s-weighted Y_lm (theta part) from the textbook Y_lm by applying
    eth f = -(d_theta - s cot - m csc) f (raising) or bar-eth (lowering) |s| times."""
    import sympy as sp
    th = sp.symbols("theta")
    ph = sp.symbols("phi", real=True)
    f = sp.simplify(sp.Ynm(l, m, th, ph).expand(func=True) * sp.exp(-sp.I * m * ph))
    cur = 0
    for _ in range(abs(s)):
        if s > 0:
            f = -(sp.diff(f, th) - cur * sp.cot(th) * f - m / sp.sin(th) * f)
            f = f / sp.sqrt((l - cur) * (l + cur + 1))
            cur += 1
        else:
            g = -(sp.diff(f, th) + cur * sp.cot(th) * f + m / sp.sin(th) * f)
            f = -g / sp.sqrt((l + cur) * (l - cur + 1))
            cur -= 1
    return sp.lambdify(th, f, "math")


@pytest.mark.parametrize("s", [-3, -2, -1, 1, 2, 3])
def test_spin_harmonics_from_eth(s):
    """Recurrence values equal eth^|s| (or bar-eth) applied symbolically to Y_lm."""
    pytest.importorskip("sympy")
    for l in range(abs(s), 6):
        for m in range(0, l + 1):
            f = _sympy_spin_Y(l, m, s)
            for th in (0.3, 1.1, 2.5):
                lam = sht.spin_lambda(8, m, s, th)
                assert abs(lam[l] - f(th)) < 1e-12, (s, l, m, th)


@pytest.mark.parametrize("s", [0, 1, 2, -2, 6])
def test_unsold_sum_rule(s):
    """sum_{m=-l}^{l} |sY_lm|^2 = (2l+1)/(4 pi) at every theta; with
    |s lambda_{l,-m}| = |-s lambda_{lm}| this needs only m >= 0."""
    lmax = 1500
    for th in (0.0011, 0.05, 0.9, 1.5707, 2.6, 3.14):
        tot = np.zeros(lmax + 1)
        for m in range(lmax + 1):
            a = sht.spin_lambda(lmax, m, s, th)
            if m == 0:
                tot += a * a
            else:
                b = sht.spin_lambda(lmax, m, -s, th)
                tot += a * a + b * b
        l = np.arange(lmax + 1)
        ok = l >= abs(s)
        # cos(theta) is only representable to 1.1e-16, which moves theta itself by
        # ~1e-16/theta^2 relative near the poles; allow for that conditioning.
        rtol = 1e-11 if min(th, pi - th) > 0.04 else 1e-9
        assert np.allclose(tot[ok], (2 * l[ok] + 1) / (4 * pi), rtol=rtol, atol=0), th


def test_orthonormal_by_quadrature():
    """2 pi int slam_lm slam_l'm sin(theta) dtheta = delta_ll' (Gauss-Legendre in cos theta)."""
    x, w = np.polynomial.legendre.leggauss(80)
    th = np.arccos(x)
    for s, m in ((0, 3), (2, 0), (2, 5), (-2, 1)):
        lam = np.array([sht.spin_lambda(40, m, s, t) for t in th])
        G = 2 * pi * (lam * w[:, None]).T @ lam
        l0 = max(abs(s), m)
        assert np.allclose(G[l0:, l0:], np.eye(41 - l0), atol=1e-12), (s, m)


@pytest.mark.parametrize("s", [0, 2, -2])
def test_theta_derivatives_exact_fourier(s):
    """slambda_lm(theta) continues to a trigonometric polynomial of degree l on the
    circle: sampling 2l+2 points, one DFT and multiplying by (ik)^j differentiates exactly."""
    for l, m in ((7, 3), (20, 0), (33, 12), (60, 41)):
        N = 2 * l + 2
        grid = (np.arange(N) + 0.5) * 2 * pi / N
        vals = np.array([sht.spin_lambda(l, m, s, t)[l] for t in grid])
        k = np.fft.fftfreq(N, 1.0 / N)
        # grid offset by half a cell: undo its phase to get the true coefficients
        c = np.fft.fft(vals) / N * np.exp(-1j * k * pi / N)
        for th in (0.2, 1.0, 2.9):
            der = sht.spin_lambda_derivs(l, m, s, 6, th)[:, l]
            for j in range(7):
                ref = np.sum(c * (1j * k) ** j * np.exp(1j * k * th)).real
                scale = max(1.0, l ** j) * np.abs(vals).max()
                assert abs(der[j] - ref) < 1e-11 * scale, (l, m, j, th)


def test_theta_derivatives_richardson_large_l():
    """Richardson-extrapolated central differences at l ~ 1000 (normalisation and
    rescaling regime), first and second derivative."""
    lmax = 1000
    for s in (0, 2):
        for m in (0, 300, 900):
            th = 0.8
            h = 2e-4
            f = lambda t: sht.spin_lambda(lmax, m, s, t)
            d1_h = (f(th + h) - f(th - h)) / (2 * h)
            d1_h2 = (f(th + h / 2) - f(th - h / 2)) / h
            d1 = (4 * d1_h2 - d1_h) / 3
            d2_h = (f(th + h) - 2 * f(th) + f(th - h)) / h ** 2
            d2_h2 = (f(th + h / 2) - 2 * f(th) + f(th - h / 2)) / (h / 2) ** 2
            d2 = (4 * d2_h2 - d2_h) / 3
            der = sht.spin_lambda_derivs(lmax, m, s, 2, th)
            sc = np.abs(f(th)).max()
            assert np.abs(der[1] - d1).max() < 2e-5 * sc * lmax
            assert np.abs(der[2] - d2).max() < 2e-5 * sc * lmax ** 2


def test_closed_form_l2():
    """Table values: Y_20, Y_21, Y_22 and 2Y_20 = sqrt(15/(32 pi)) sin^2 theta."""
    th = 0.77
    c, s = np.cos(th), np.sin(th)
    lam = [sht.spin_lambda(2, m, 0, th)[2] for m in range(3)]
    assert np.isclose(lam[0], sqrt(5 / (16 * pi)) * (3 * c * c - 1), rtol=1e-14)
    assert np.isclose(lam[1], -sqrt(15 / (8 * pi)) * s * c, rtol=1e-14)
    assert np.isclose(lam[2], sqrt(15 / (32 * pi)) * s * s, rtol=1e-14)
    assert np.isclose(sht.spin_lambda(2, 0, 2, th)[2], sqrt(15 / (32 * pi)) * s * s, rtol=1e-14)
    assert np.isclose(sht.spin_lambda(2, 0, -2, th)[2], sqrt(15 / (32 * pi)) * s * s, rtol=1e-14)


def test_tiny_seed_no_underflow_trouble():
    """Near the pole at large m the seed is ~1e-3000; values must be finite, and
    zero (not NaN) where they are below the double range."""
    lam = sht.spin_lambda(4096, 4000, 2, 0.0004)
    assert np.all(np.isfinite(lam))
    assert np.all(lam == 0.0)
    lam = sht.spin_lambda(4096, 100, 0, 0.03)
    assert np.all(np.isfinite(lam)) and np.abs(lam).max() > 0.1
