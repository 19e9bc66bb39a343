"""Full-sky pixel-relative Taylor lensing, plain FP64 (oracle; test infrastructure only).

Follows the paper's steps in order (Naess & Louis 2013):
  1. deflection alpha = grad(phi) at every pixel centre           (Sec. I, Eqs. 1-2; Sec. II.A)
  2. displaced position x' = x + alpha                             (Sec. II.A)
  3. expansion point: the pixel containing x' via ang2pix, its
     centre x0' via pix2ang, offset Delta alpha = x' - x0'         (Sec. II.B)
  4. derivative maps d_theta^j d_phi^k s for s in {T, Q, U}, j+k <= n
  5. Taylor sum per component, Eq. 4                               (Sec. II.B)
  6. polarisation rotation R from parallel transport               (Eq. 2; Sec. II.B)

Readings where the paper is silent (each listed in the design notes):
  - derivatives are the exact coordinate derivatives of the band-limited field,
    the expansion variables are (Delta theta, Delta phi);
  - x' is the end point of the geodesic leaving x in the direction of alpha
    with length |alpha| (the parallel-transport form of the displacement);
  - Delta phi is wrapped into [-pi, pi);
  - R multiplies Q + iU by exp(-2 i beta), beta the angle, measured from
    e_theta towards e_phi at x', of e_theta(x) carried to x' by parallel
    transport along that geodesic;
  - "order n" means total degree j + k <= n; order 0 is the nearest-pixel lookup.
"""
from __future__ import annotations

from math import factorial

import numpy as np

from . import healpix as hp
from . import sht


def map_index(j: int, k: int) -> int:
    """Position of d_theta^j d_phi^k among the (n+1)(n+2)/2 maps of one field,
    ordered by total degree and then by j."""
    N = j + k
    return N * (N + 1) // 2 + j


def derivative_pairs(order: int):
    return [(j, N - j) for N in range(order + 1) for j in range(N + 1)]


# ---------------------------------------------------------------------------
# ring synthesis: D(theta_r, phi_p) = Re[ G_0 + 2 sum_{m>0} G_m e^{i m phi_p} ],
# G_m = (i m)^k F^j_m(theta_r), evaluated on the ring's nphi equally spaced
# longitudes by folding m modulo nphi and one inverse DFT (library FFT).

def ring_synthesis(F: np.ndarray, nphi: int, phi0: float, jk_list):
    """F: [nder+1, mmax+1] complex coefficients of one ring. Returns [len(jk_list), nphi]."""
    mmax = F.shape[1] - 1
    m = np.arange(mmax + 1)
    w = np.where(m == 0, 1.0, 2.0)
    phase = np.exp(1j * m * phi0)
    out = np.empty((len(jk_list), nphi))
    for idx, (j, k) in enumerate(jk_list):
        G = (1j * m) ** k * F[j] * w * phase
        B = np.zeros(nphi, dtype=np.complex128)
        np.add.at(B, m % nphi, G)
        out[idx] = (np.fft.ifft(B) * nphi).real
    return out


def derivative_maps(nside: int, lmax: int, order: int, alm_T=None, alm_E=None, alm_B=None,
                    jk_list=None, nthreads=None):
    """All derivative maps d_theta^j d_phi^k s at every pixel centre (RING order).

    Returns dict field -> array [n_maps, Npix] in map_index order (or jk_list order).
    """
    tab = hp.ring_table(nside)
    jk = derivative_pairs(order) if jk_list is None else list(jk_list)
    nder = max(j for j, _ in jk)
    F = sht.ring_coeffs(lmax, nder, tab["theta"], alm_T, alm_E, alm_B, nthreads=nthreads)
    out = {f: np.empty((len(jk), hp.npix(nside))) for f in F}
    for r in range(tab["theta"].size):
        a, n = tab["first"][r], tab["nphi"][r]
        for f in F:
            out[f][:, a:a + n] = ring_synthesis(F[f][r], int(n), tab["phi0"][r], jk)
    return out


def deflection(nside: int, lmax: int, alm_phi, nthreads=None):
    """alpha = (d_theta phi, d_phi phi / sin theta) at every pixel centre (Sec. I)."""
    tab = hp.ring_table(nside)
    maps = derivative_maps(nside, lmax, 1, alm_T=alm_phi, jk_list=[(1, 0), (0, 1)],
                           nthreads=nthreads)["T"]
    sint = np.repeat(tab["sint"], tab["nphi"])
    return maps[0], maps[1] / sint


# ---------------------------------------------------------------------------
# geometry

def basis(theta, phi):
    """Unit position vector and the (e_theta, e_phi) tangent basis."""
    st, ct, sp, cp = np.sin(theta), np.cos(theta), np.sin(phi), np.cos(phi)
    n = np.stack([st * cp, st * sp, ct], axis=-1)
    et = np.stack([ct * cp, ct * sp, -st], axis=-1)
    ep = np.stack([-sp, cp, np.zeros_like(sp)], axis=-1)
    return n, et, ep


def basis_zs(z, s, phi):
    sp, cp = np.sin(phi), np.cos(phi)
    n = np.stack([s * cp, s * sp, z], axis=-1)
    et = np.stack([z * cp, z * sp, -s], axis=-1)
    ep = np.stack([-sp, cp, np.zeros_like(sp)], axis=-1)
    return n, et, ep


def displace(z, s, phi, a_th, a_ph):
    """Geodesic of length |alpha| leaving (theta, phi) along alpha.

    Returns n' (unit vector of x'), the unit direction u of alpha at x, and d = |alpha|.
    """
    n, et, ep = basis_zs(z, s, phi)
    d = np.hypot(a_th, a_ph)
    with np.errstate(invalid="ignore", divide="ignore"):
        ut = np.where(d > 0, a_th / np.where(d > 0, d, 1.0), 1.0)
        up = np.where(d > 0, a_ph / np.where(d > 0, d, 1.0), 0.0)
    u = ut[..., None] * et + up[..., None] * ep
    n2 = np.cos(d)[..., None] * n + np.sin(d)[..., None] * u
    return n2, u, n, et, d


def rotate_about(v, axis, ang):
    """Rodrigues rotation of vectors v about unit axis by angle ang (right-handed)."""
    c, s = np.cos(ang)[..., None], np.sin(ang)[..., None]
    return v * c + np.cross(axis, v) * s + axis * np.sum(axis * v, axis=-1, keepdims=True) * (1 - c)


def transport_angle(n, u, et, d, theta2, phi2):
    """beta: angle at x' (from e_theta towards e_phi) of e_theta(x) parallel-transported
    along the geodesic x -> x'. Transport along a great circle is the rotation about
    its pole a = n x u by the arc length d."""
    axis = np.cross(n, u)
    t = rotate_about(et, axis, d)
    _, et2, ep2 = basis(theta2, phi2)
    return np.arctan2(np.sum(t * ep2, axis=-1), np.sum(t * et2, axis=-1))


def wrap_pi(x):
    """Wrap into [-pi, pi)."""
    return np.mod(x + np.pi, 2.0 * np.pi) - np.pi


def target_point(theta, z, s, phi, a_th, a_ph, naive=False):
    """The displaced position x' of Sec. II.A and the geodesic pieces R uses.

    Default: the end of the geodesic of length |alpha| leaving x along alpha.
    naive=True: the paper's alternative, coordinate addition theta' = theta + a_theta,
    phi' = phi + a_phi / sin(theta); a point carried past a pole continues on the
    other side (theta' -> -theta' or 2 pi - theta', phi' -> phi' + pi). The
    rotation R keeps the geodesic transport angle in both cases (beta at the geodesic
    end point). d = 0 returns x exactly. Returns theta', phi', z', sin(theta') and the
    pieces of R: (n, u, e_theta, d, theta_g, phi_g), (theta_g, phi_g) the geodesic end."""
    n2, u, n, et, d = displace(z, s, phi, a_th, a_ph)
    still = d == 0
    theta_g = np.where(still, theta, np.arctan2(np.hypot(n2[:, 0], n2[:, 1]), n2[:, 2]))
    phi_g = np.where(still, phi, np.mod(np.arctan2(n2[:, 1], n2[:, 0]), 2.0 * np.pi))
    if naive:
        theta2 = theta + a_th
        with np.errstate(divide="ignore", invalid="ignore"):
            phi2 = phi + np.where(s > 0, a_ph / np.where(s > 0, s, 1.0), 0.0)
        north, south = theta2 < 0.0, theta2 > np.pi
        theta2 = np.where(north, -theta2, np.where(south, 2.0 * np.pi - theta2, theta2))
        phi2 = np.mod(np.where(north | south, phi2 + np.pi, phi2), 2.0 * np.pi)
        z2, s2 = np.cos(theta2), np.sin(theta2)
    else:
        z2 = np.clip(n2[:, 2], -1.0, 1.0)
        s2 = np.hypot(n2[:, 0], n2[:, 1])
        theta2 = np.arctan2(s2, n2[:, 2])
        phi2 = np.mod(np.arctan2(n2[:, 1], n2[:, 0]), 2.0 * np.pi)
    theta2 = np.where(still, theta, theta2)
    phi2 = np.where(still, phi, phi2)
    z2 = np.where(still, z, z2)
    s2 = np.where(still, s, s2)
    return theta2, phi2, z2, s2, (n, u, et, d, theta_g, phi_g)


def expansion_point(nside, pix, theta2, phi2, z2, s2, theta_p, phi_p, at_pixel=False):
    """The expansion pixel q and the offsets (dth, dph) of Eq. 4: by default q is the
    pixel containing x' (Sec. II.B); at_pixel=True expands about the output pixel
    itself, q = p, the plain Taylor series about the undisplaced point of Sec. I
    (Eq. 3a). dph is wrapped into [-pi, pi)."""
    if at_pixel:
        q = np.asarray(pix, dtype=np.int64)
        return q, theta2 - theta_p, wrap_pi(phi2 - phi_p)
    q = hp.ang2pix(nside, z2, s2, phi2)
    th_q, ph_q = hp.pix2ang(nside, q)
    return q, theta2 - th_q, wrap_pi(phi2 - ph_q)


# ---------------------------------------------------------------------------

def taylor_sum(D_at_q: np.ndarray, dth, dph, order: int):
    """Eq. 4: sum over total degree N <= n and j <= N of
    dth^j dph^(N-j) / (j! (N-j)!) * D_{j, N-j}(x0')."""
    out = np.zeros_like(dth)
    for N in range(order + 1):
        for j in range(N + 1):
            k = N - j
            out = out + dth ** j * dph ** k / (factorial(j) * factorial(k)) * D_at_q[map_index(j, k)]
    return out


def lens(nside: int, lmax: int, order: int, alm_T, alm_E=None, alm_B=None, alm_phi=None,
         rotate: bool = True, nthreads=None, return_aux: bool = False, naive: bool = False,
         at_pixel: bool = False, lmax_phi=None):
    """Lensed T (and Q, U) maps in RING order, FP64 (naive, at_pixel: see target_point
    and expansion_point). lmax_phi: the potential's own band limit (Sec. II.A: the
    gradient map is taken to min(8 Nside, 10000)); alm_phi is then in that layout."""
    tab = hp.ring_table(nside)
    npx = hp.npix(nside)
    pix = np.arange(npx)
    ring, jidx = hp.pix2ring(nside, pix)
    z = tab["z"][ring - 1]
    s = tab["sint"][ring - 1]
    phi = tab["phi0"][ring - 1] + 2.0 * np.pi * jidx / tab["nphi"][ring - 1]
    # 1. deflection
    if alm_phi is None:
        a_th = np.zeros(npx)
        a_ph = np.zeros(npx)
    else:
        a_th, a_ph = deflection(nside, lmax if lmax_phi is None else lmax_phi, alm_phi, nthreads=nthreads)
    # 2. displaced position (zero displacement: x' = x exactly)
    theta_p = tab["theta"][ring - 1]
    theta2, phi2, z2, s2, (n, u, et, d, theta_g, phi_g) = target_point(theta_p, z, s, phi, a_th, a_ph, naive)
    still = d == 0
    # 3. expansion point
    q, dth, dph = expansion_point(nside, pix, theta2, phi2, z2, s2, theta_p, phi, at_pixel)
    # 4. derivative maps
    maps = derivative_maps(nside, lmax, order, alm_T, alm_E, alm_B, nthreads=nthreads)
    # 5. Taylor sum
    out = {f: taylor_sum(maps[f][:, q], dth, dph, order) for f in maps}
    # 6. rotation
    beta = np.zeros(npx)
    if "Q" in out and rotate:
        beta = np.where(still, 0.0, transport_angle(n, u, et, d, theta_g, phi_g))
        P = (out["Q"] + 1j * out["U"]) * np.exp(-2j * beta)
        out["Q"], out["U"] = P.real, P.imag
    if return_aux:
        out["aux"] = dict(q=q, dth=dth, dph=dph, beta=beta, a_th=a_th, a_ph=a_ph,
                          theta2=theta2, phi2=phi2)
    return out


def exact_at(lmax: int, theta, phi, alm_T=None, alm_E=None, alm_B=None, nthreads=None):
    """Brute force: the unlensed fields summed directly at arbitrary points,
    T(x) = sum_lm T_lm Y_lm(x), Q +- iU = -sum (E +- iB) +-2Y_lm."""
    F = sht.ring_coeffs(lmax, 0, theta, alm_T, alm_E, alm_B, nthreads=nthreads)
    return {f: sht.point_sum(F[f], phi, 0, 0, nthreads=nthreads) for f in F}


def lens_exact(nside: int, lmax: int, alm_T, alm_E=None, alm_B=None, alm_phi=None, pix=None,
               nthreads=None, lmax_phi=None):
    """Exact Born remap (Eqs. 1-2) at the given pixels by direct spherical-harmonic
    sums at the displaced positions, with the same rotation R (lmax_phi as in lens)."""
    tab = hp.ring_table(nside)
    npx = hp.npix(nside)
    pix = np.arange(npx) if pix is None else np.asarray(pix)
    ring, jidx = hp.pix2ring(nside, pix)
    z = tab["z"][ring - 1]
    s = tab["sint"][ring - 1]
    phi = tab["phi0"][ring - 1] + 2.0 * np.pi * jidx / tab["nphi"][ring - 1]
    a_th, a_ph = deflection_at(lmax if lmax_phi is None else lmax_phi, alm_phi, tab["theta"][ring - 1], phi, s,
                               nthreads)
    n2, u, n, et, d = displace(z, s, phi, a_th, a_ph)
    theta2 = np.arctan2(np.hypot(n2[:, 0], n2[:, 1]), n2[:, 2])
    phi2 = np.mod(np.arctan2(n2[:, 1], n2[:, 0]), 2.0 * np.pi)
    out = exact_at(lmax, theta2, phi2, alm_T, alm_E, alm_B, nthreads)
    if "Q" in out:
        beta = np.where(d == 0, 0.0, transport_angle(n, u, et, d, theta2, phi2))
        P = (out["Q"] + 1j * out["U"]) * np.exp(-2j * beta)
        out["Q"], out["U"] = P.real, P.imag
    return out


def _ring_coeffs_unique(lmax, nder, theta, nthreads=None, **alm):
    """ring_coeffs at each point's colatitude, each distinct colatitude computed once
    (points on one ring share it exactly)."""
    uth, inv = np.unique(np.asarray(theta, dtype=np.float64), return_inverse=True)
    F = sht.ring_coeffs(lmax, nder, uth, nthreads=nthreads, **alm)
    return {f: v[inv] for f, v in F.items()}


def deflection_at(lmax, alm_phi, theta, phi, sint, nthreads=None):
    if alm_phi is None:
        return np.zeros_like(theta), np.zeros_like(theta)
    F = _ring_coeffs_unique(lmax, 1, theta, nthreads, alm_T=alm_phi)["T"]
    a_th = sht.point_sum(F, phi, 1, 0, nthreads=nthreads)
    a_ph = sht.point_sum(F, phi, 0, 1, nthreads=nthreads) / sint
    return a_th, a_ph


def lens_at_pixels(nside: int, lmax: int, order: int, pix, alm_T, alm_E=None, alm_B=None,
                   alm_phi=None, rotate: bool = True, nthreads=None, naive: bool = False,
                   at_pixel: bool = False, lmax_phi=None):
    """The same algorithm as `lens`, evaluated only at the given output pixels:
    derivative values at each expansion pixel come from direct Fourier sums
    instead of ring FFTs (used for sampled checks at full size)."""
    tab = hp.ring_table(nside)
    pix = np.asarray(pix, dtype=np.int64)
    ring, jidx = hp.pix2ring(nside, pix)
    z = tab["z"][ring - 1]
    s = tab["sint"][ring - 1]
    phi = tab["phi0"][ring - 1] + 2.0 * np.pi * jidx / tab["nphi"][ring - 1]
    a_th, a_ph = deflection_at(lmax if lmax_phi is None else lmax_phi, alm_phi, tab["theta"][ring - 1], phi, s,
                               nthreads)
    theta_p = tab["theta"][ring - 1]
    theta2, phi2, z2, s2, (n, u, et, d, theta_g, phi_g) = target_point(theta_p, z, s, phi, a_th, a_ph, naive)
    still = d == 0
    q, dth, dph = expansion_point(nside, pix, theta2, phi2, z2, s2, theta_p, phi, at_pixel)
    th_q, ph_q = hp.pix2ang(nside, q)
    F = _ring_coeffs_unique(lmax, order, th_q, nthreads, alm_T=alm_T, alm_E=alm_E, alm_B=alm_B)
    out = {}
    for f in F:
        D = np.stack([sht.point_sum(F[f], ph_q, j, k, nthreads=nthreads)
                      for (j, k) in derivative_pairs(order)])
        out[f] = taylor_sum(D, dth, dph, order)
    if "Q" in out and rotate:
        beta = np.where(still, 0.0, transport_angle(n, u, et, d, theta_g, phi_g))
        P = (out["Q"] + 1j * out["U"]) * np.exp(-2j * beta)
        out["Q"], out["U"] = P.real, P.imag
    out["aux"] = dict(q=q, dth=dth, dph=dph, a_th=a_th, a_ph=a_ph)
    return out


# ---------------------------------------------------------------------------
# analysis side (Sec. III: the lensed maps are measured through power spectra)

def map2alm(nside: int, lmax: int, T, Q=None, U=None):
    """a_lm = (4 pi / Npix) sum_p s(p) conj(sY_lm(p)) with uniform weights (healpy's
    map2alm without iterations), written out as direct sums: per ring the weighted
    Fourier sums over its pixels, then the spin-weighted lambda_lm of the ring.
    Spin 2 in the HEALPix convention Q +- iU = -sum (E +- iB) +-2Y_lm:
    E = -(X+ + X-)/2, B = i (X+ - X-)/2 with X+- = sum w (Q +- iU) conj(+-2Y)."""
    tab = hp.ring_table(nside)
    w = 4.0 * np.pi / hp.npix(nside)
    na = (lmax + 1) * (lmax + 2) // 2
    out = {"T": np.zeros(na, complex)}
    pol = Q is not None
    if pol:
        out["E"] = np.zeros(na, complex)
        out["B"] = np.zeros(na, complex)
    ms = np.arange(lmax + 1)
    for r in range(len(tab["nphi"])):
        n, f0 = int(tab["nphi"][r]), int(tab["first"][r])
        ph = tab["phi0"][r] + 2.0 * np.pi * np.arange(n) / n
        e = np.exp(-1j * np.outer(ms, ph))  # [m, p]
        th = tab["theta"][r]
        ft = w * (e @ np.asarray(T[f0:f0 + n], float))
        if pol:
            p = np.asarray(Q[f0:f0 + n], float) + 1j * np.asarray(U[f0:f0 + n], float)
            fp, fm = w * (e @ p), w * (e @ np.conj(p))
        for m in range(lmax + 1):
            blk = slice(m * (2 * lmax + 1 - m) // 2 + m, m * (2 * lmax + 1 - m) // 2 + lmax + 1)  # l = m..lmax
            out["T"][blk] += ft[m] * sht.spin_lambda(lmax, m, 0, th)[m:]
            if pol:
                xp = fp[m] * sht.spin_lambda(lmax, m, 2, th)[m:]
                xm = fm[m] * sht.spin_lambda(lmax, m, -2, th)[m:]
                out["E"][blk] += -0.5 * (xp + xm)
                out["B"][blk] += 0.5j * (xp - xm)
    for f in out:  # m = 0 coefficients of a real field are real
        out[f][:lmax + 1] = out[f][:lmax + 1].real
    return out


def anafast(lmax: int, alm_x, alm_y=None):
    """C_l = (1/(2l+1)) sum_{m=-l..l} Re(x_lm conj(y_lm)) for real fields."""
    y = alm_x if alm_y is None else alm_y
    cl = np.zeros(lmax + 1)
    for m in range(lmax + 1):
        blk = slice(m * (2 * lmax + 1 - m) // 2 + m, m * (2 * lmax + 1 - m) // 2 + lmax + 1)  # l = m..lmax
        v = (alm_x[blk] * np.conj(y[blk])).real
        cl[m:] += v if m == 0 else 2.0 * v
    return cl / (2.0 * np.arange(lmax + 1) + 1.0)
