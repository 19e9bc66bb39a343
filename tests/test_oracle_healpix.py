"""Pins for the oracle's HEALPix RING geometry (Gorski et al. 2005; the paper uses
healpy's ang2pix / pix2ang, Sec. II.B)."""
import numpy as np
import pytest

import oracle.healpix as hp


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 32, 64])
def test_round_trip_every_pixel(nside):
    p = np.arange(hp.npix(nside))
    th, ph = hp.pix2ang(nside, p)
    assert np.array_equal(hp.ang2pix_theta(nside, th, ph), p)


@pytest.mark.parametrize("nside", [1, 2, 8, 64])
def test_ring_structure(nside):
    tab = hp.ring_table(nside)
    n = nside
    assert tab["nphi"].sum() == 12 * n * n
    assert len(tab["nphi"]) == 4 * n - 1
    i = np.arange(1, 4 * n)
    inorth = np.minimum(i, 4 * n - i)
    assert np.array_equal(tab["nphi"], np.where(inorth < n, 4 * inorth, 4 * n))
    # first pixel of ring i+1 = first of ring i + nphi_i
    assert np.array_equal(tab["first"][1:], tab["first"][:-1] + tab["nphi"][:-1])
    # belt rings are equally spaced in z by 2/(3N); z is antisymmetric about the equator
    belt = (i >= n) & (i <= 3 * n)
    dz = np.diff(tab["z"][belt])
    assert np.allclose(dz, -2.0 / (3 * n), rtol=0, atol=1e-15)
    assert np.allclose(tab["z"], -tab["z"][::-1], atol=1e-15)


def test_nside1_base_pixels():
    th, ph = hp.pix2ang(1, np.arange(12))
    z = np.cos(th)
    assert np.allclose(z[:4], 2 / 3) and np.allclose(z[4:8], 0, atol=1e-15) and np.allclose(z[8:], -2 / 3)
    assert ph[4] == 0.0
    assert np.allclose(ph[:4], np.pi / 4 + np.arange(4) * np.pi / 2)


@pytest.mark.parametrize("nside", [1, 4, 16])
def test_equal_area_monte_carlo(nside):
    """Uniform points land in every pixel equally often (equal-area cells) --
    only true if all the cell boundaries are right."""
    rng = np.random.default_rng(7)
    npx = hp.npix(nside)
    M = 4000 * npx
    z = rng.uniform(-1, 1, M)
    phi = rng.uniform(0, 2 * np.pi, M)
    cnt = np.bincount(hp.ang2pix(nside, z, np.sqrt(1 - z * z), phi), minlength=npx)
    expect = M / npx
    chi2 = np.sum((cnt - expect) ** 2 / expect)
    dof = npx - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof), chi2


@pytest.mark.parametrize("nside", [4, 32])
def test_belt_cells_are_the_rhombi(nside):
    """In the belt, (t, z) with t = 2 phi/pi: the cell of centre (t_c, z_c) is
    2N|t - t_c| + (3N/2)|z - z_c| <= 1 (Gorski et al. 2005, Sec. 4)."""
    rng = np.random.default_rng(3)
    z = rng.uniform(-0.6, 0.6, 20000)
    phi = rng.uniform(0, 2 * np.pi, 20000)
    p = hp.ang2pix(nside, z, np.sqrt(1 - z * z), phi)
    thc, phc = hp.pix2ang(nside, p)
    zc = np.cos(thc)
    dt = (phi - phc) * 2 / np.pi
    dt = (dt + 2) % 4 - 2
    lhs = 2 * nside * np.abs(dt) + 1.5 * nside * np.abs(z - zc)
    assert lhs.max() <= 1 + 1e-9


@pytest.mark.parametrize("nside", [8, 64])
def test_containing_pixel_is_close(nside):
    """The pixel containing a point has its centre within the largest cell radius."""
    rng = np.random.default_rng(5)
    z = rng.uniform(-1, 1, 20000)
    phi = rng.uniform(0, 2 * np.pi, 20000)
    s = np.sqrt(1 - z * z)
    p = hp.ang2pix(nside, z, s, phi)
    thc, phc = hp.pix2ang(nside, p)
    cosd = z * np.cos(thc) + s * np.sin(thc) * np.cos(phi - phc)
    d = np.arccos(np.clip(cosd, -1, 1))
    # max pixel radius is below ~ 1.4 x the mean cell size
    assert d.max() < 1.4 * np.sqrt(4 * np.pi / hp.npix(nside))


@pytest.mark.parametrize("nside", [1, 2, 8, 64, 1024])
def test_pixel_centres_at_half_integer_cell_coordinates(nside):
    """Every pixel centre sits at half-integers of the cell coordinates that bound the
    cells (Gorski et al. 2005): in the belt x1 = N(t + 1/2) - (3/4) N z = idx + (sh + i - N)/2
    and x2 = N(t + 1/2) + (3/4) N z = idx + (3N + sh - i)/2 (ring i, half-pixel shift sh);
    in a cap, with i the ring's distance from its pole, N sqrt(3 (1 - |z|)) = i and
    frac(t) = (k + 1/2)/i with k = idx mod i. The float gather's pixel lookup works in
    increments from these exact values."""
    n = nside
    tab = hp.ring_table(n)
    p = np.arange(hp.npix(n))
    ring, idx = hp.pix2ring(n, p)
    th, ph = hp.pix2ang(n, p)
    z = np.cos(th)
    t = ph * (2.0 / np.pi)
    sh = (tab["phi0"][ring - 1] != 0).astype(np.int64)
    belt = (ring >= n) & (ring <= 3 * n)
    x1 = n * (0.5 + t) - 0.75 * n * z
    x2 = n * (0.5 + t) + 0.75 * n * z
    tol = 1e-9 * 4 * n
    assert np.all(((sh + ring - n) % 2 == 1)[belt])
    assert np.allclose(x1[belt], (idx + (sh + ring - n) / 2.0)[belt], rtol=0, atol=tol)
    assert np.allclose(x2[belt], (idx + (3 * n + sh - ring) / 2.0)[belt], rtol=0, atol=tol)
    cap = ~belt
    i = np.where(ring < n, ring, 4 * n - ring)[cap]
    omz = tab["omz"][ring - 1][cap]
    assert np.allclose(n * np.sqrt(3.0 * omz), i, rtol=0, atol=tol)
    k = idx[cap] % i
    assert np.allclose(t[cap] - np.floor(t[cap]), (k + 0.5) / i, rtol=0, atol=1e-12)
