"""HEALPix RING-scheme geometry in FP64 (oracle; test infrastructure only).

Restated from the pixel-boundary description of Gorski et al. (2005, ApJ 622, 759);
the paper itself only calls healpy's ang2pix / pix2ang (Sec. II.B).

Rings i = 1 .. 4 Nside - 1, counted from the north pole:
  north cap  i <  Nside : z = 1 - i^2/(3 Nside^2), 4 i pixels, phi_j = pi/(2i) (j + 1/2)
  belt  Nside <= i <= 3 Nside : z = 4/3 - 2 i/(3 Nside), 4 Nside pixels,
        phi_j = pi/(2 Nside) (j + 1/2) when i - Nside is even, pi/(2 Nside) j otherwise
  south cap: mirror image of the north cap.
"""
from __future__ import annotations

import numpy as np


def npix(nside: int) -> int:
    return 12 * nside * nside


def ring_table(nside: int):
    """Per ring (index 0 = ring 1): z, 1-|z| (exact in the caps), theta, sin(theta),
    nphi, phi0 (longitude of the ring's first pixel), first pixel index."""
    n = nside
    nr = 4 * n - 1
    i = np.arange(1, nr + 1, dtype=np.int64)
    inorth = np.minimum(i, 4 * n - i)  # ring number counted from the nearer pole
    z = np.empty(nr)
    omz = np.empty(nr)  # 1 - |z|
    nphi = np.empty(nr, dtype=np.int64)
    phi0 = np.empty(nr)
    first = np.empty(nr, dtype=np.int64)
    cap = inorth < n
    # caps
    ic = inorth[cap]
    omz[cap] = ic.astype(np.float64) ** 2 / (3.0 * n * n)
    nphi[cap] = 4 * ic
    phi0[cap] = np.pi / (2.0 * ic) * 0.5
    # belt
    ib = i[~cap]
    zb = 4.0 / 3.0 - 2.0 * ib / (3.0 * n)
    omz[~cap] = 1.0 - np.abs(zb)
    nphi[~cap] = 4 * n
    shifted = ((ib - n) % 2) == 0
    phi0[~cap] = np.where(shifted, np.pi / (2.0 * n) * 0.5, 0.0)
    sign = np.where(i <= 2 * n, 1.0, -1.0)
    z = sign * (1.0 - omz)
    z[~cap] = zb
    # first pixel of each ring
    ncap = 2 * n * (n - 1)
    north = i < n
    south = i > 3 * n
    belt = ~(north | south)
    first[north] = 2 * i[north] * (i[north] - 1)
    first[belt] = ncap + (i[belt] - n) * 4 * n
    isouth = 4 * n - i[south]
    first[south] = npix(n) - 2 * isouth * (isouth + 1)
    # theta from 1-|z| without cancellation: sin^2(theta/2) = (1-z)/2
    sin_half = np.sqrt(omz / 2.0)
    theta_pole = 2.0 * np.arcsin(sin_half)  # distance to the nearer pole
    theta = np.where(sign > 0, theta_pole, np.pi - theta_pole)
    sint = np.sqrt(omz * (2.0 - omz))
    return dict(z=z, omz=omz, theta=theta, sint=sint, nphi=nphi, phi0=phi0, first=first)


def pix2ring(nside: int, pix):
    """Ring number (1-based) and index within the ring of each pixel."""
    n = nside
    pix = np.asarray(pix, dtype=np.int64)
    ncap = 2 * n * (n - 1)
    ring = np.empty_like(pix)
    j = np.empty_like(pix)
    north = pix < ncap
    south = pix >= npix(n) - ncap
    belt = ~(north | south)
    # north cap: first pixel of ring i is 2 i (i-1)
    p = pix[north]
    i = ((1 + np.sqrt(1.0 + 2.0 * p)) // 2).astype(np.int64)
    i = np.where(2 * i * (i - 1) > p, i - 1, i)
    i = np.where(2 * (i + 1) * i <= p, i + 1, i)
    ring[north] = i
    j[north] = p - 2 * i * (i - 1)
    # belt
    p = pix[belt] - ncap
    ring[belt] = p // (4 * n) + n
    j[belt] = p % (4 * n)
    # south cap, mirrored: pixel Npix-1-p counted from the south pole
    p = npix(n) - 1 - pix[south]
    i = ((1 + np.sqrt(1.0 + 2.0 * p)) // 2).astype(np.int64)
    i = np.where(2 * i * (i - 1) > p, i - 1, i)
    i = np.where(2 * (i + 1) * i <= p, i + 1, i)
    ring[south] = 4 * n - i
    j[south] = 4 * i - 1 - (p - 2 * i * (i - 1))
    return ring, j


def pix2ang(nside: int, pix):
    """Centre (theta, phi) of each pixel."""
    tab = ring_table(nside)
    ring, j = pix2ring(nside, pix)
    r = ring - 1
    theta = tab["theta"][r]
    phi = tab["phi0"][r] + 2.0 * np.pi * j / tab["nphi"][r]
    return theta, phi


def ang2pix(nside: int, z, s, phi):
    """Pixel containing the point with cos(theta) = z, sin(theta) = s >= 0, longitude phi.

    Belt (|z| <= 2/3): pixel edges are the lines N(t + 1/2) -+ (3/4) N z in Z,
    with t = 2 phi / pi.  Caps: with tmp = N sqrt(3 (1 - |z|)) and tp = frac(t),
    edges are tp*tmp in Z and (1-tp)*tmp in Z; the ring is the number of edges
    crossed from the pole.
    """
    n = nside
    z = np.asarray(z, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    za = np.abs(z)
    t = np.mod(phi, 2.0 * np.pi) * (2.0 / np.pi)
    t = np.where(t >= 4.0, t - 4.0, t)
    out = np.empty(z.shape, dtype=np.int64)
    belt = za <= 2.0 / 3.0
    # ---- belt
    zb, tb = z[belt], t[belt]
    a = n * (0.5 + tb)
    b = 0.75 * n * zb
    jp = np.floor(a - b).astype(np.int64)  # ascending edge index
    jm = np.floor(a + b).astype(np.int64)  # descending edge index
    ir = n + 1 + jp - jm  # 1 .. 2N+1, ring N-1+ir
    kshift = 1 - (ir & 1)
    ip = (jp + jm - n + kshift + 1) // 2
    ip = np.mod(ip, 4 * n)
    out[belt] = 2 * n * (n - 1) + (ir - 1) * 4 * n + ip
    # ---- caps
    zc, sc, tc = z[~belt], s[~belt], t[~belt]
    omz = sc * sc / (1.0 + np.abs(zc))  # 1 - |z| without cancellation
    tp = tc - np.floor(tc)
    tmp = n * np.sqrt(3.0 * omz)
    jp = np.floor(tp * tmp).astype(np.int64)
    jm = np.floor((1.0 - tp) * tmp).astype(np.int64)
    ir = jp + jm + 1  # ring counted from the pole
    ip = np.floor(tc * ir).astype(np.int64)
    ip = np.mod(ip, 4 * ir)
    north = zc > 0
    out_c = np.where(north, 2 * ir * (ir - 1) + ip, npix(n) - 2 * ir * (ir + 1) + ip)
    out[~belt] = out_c
    return out


def ang2pix_theta(nside: int, theta, phi):
    theta = np.asarray(theta, dtype=np.float64)
    return ang2pix(nside, np.cos(theta), np.sin(theta), phi)


def check_pixels(nside: int, seed: int = 11, n_random: int = 128, per_ring: int = 64, cap_rings: int = 4):
    """Output pixels for sampled checks at full size (test infrastructure): every
    pixel of the first and last `cap_rings` rings, `per_ring` evenly spaced pixels
    on the last cap ring and the first belt ring of each hemisphere and on the
    equator, and `n_random` seeded random pixels. Sorted, unique, RING indices."""
    n = int(nside)
    tab = ring_table(n)
    first, nphi = tab["first"], tab["nphi"]
    nr = 4 * n - 1
    pix = []
    for i in list(range(1, min(cap_rings, nr) + 1)) + list(range(max(nr - cap_rings + 1, 1), nr + 1)):
        pix.append(first[i - 1] + np.arange(nphi[i - 1]))
    for i in sorted({max(n - 1, 1), n, 2 * n, 3 * n, min(3 * n + 1, nr)}):
        k = min(per_ring, int(nphi[i - 1]))
        pix.append(first[i - 1] + (np.arange(k) * nphi[i - 1]) // k)
    rng = np.random.default_rng(seed)
    pix.append(rng.choice(npix(n), size=min(n_random, npix(n)), replace=False))
    return np.unique(np.concatenate(pix).astype(np.int64))
