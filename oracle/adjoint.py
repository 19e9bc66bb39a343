"""Adjoint of full-sky Taylor lensing, plain FP64 (oracle; test infrastructure only).

The forward map is oracle.lens (Naess & Louis 2013, Sec. II; Eq. 4 and R of Eq. 2).
For upstream map gradients g_T, g_Q, g_U (dL/dT'(p) etc.) this returns the
coefficient gradients dL/dRe + i dL/dIm of the stored a_lm (m >= 0) of T, E, B
and the lensing potential, with the expansion pixel q(p) held fixed (the map is
piecewise smooth in the deflection; the pixel choice is constant between jumps).

Steps, each the transpose of a forward step:
  R:          (Q', U') = R(beta) (Q~, U~)        -> (gQ~, gU~) = R(beta)^T (gQ, gU)
  Eq. 4:      s~(p) = sum w_jk(D(p)) D_jk(q(p))  -> Dbar_jk[q] += w_jk gs~;  dL/dDelta from
                                                    the derivative of the polynomial
  geometry:   Delta(alpha), beta(alpha) at fixed q -> gradient wrt alpha through their
                                                    Jacobian (Richardson central differences)
  synthesis:  D_jk = Re sum_m w_m (im)^k F^j_m e^{i m phi} -> Fbar^j_m = w_m sum_k (-im)^k
                                                    sum_i Dbar_jk(i) e^{-i m phi_i} (library FFT)
  Legendre:   F = sum_l a_l lambda                 -> abar (sht.ring_adjoint)
  deflection: alpha = (D^phi_10, D^phi_01 / sin th) -> the same two transposes for phi.
"""
from __future__ import annotations

from math import factorial

import numpy as np

from . import healpix as hp
from . import lens as L
from . import sht


def ring_synthesis_adjoint(Dbar: dict, nside: int, nder: int, mmax: int):
    """Dbar: {(j, k): [Npix]} -> Fbar [nrings, nder+1, mmax+1] complex."""
    tab = hp.ring_table(nside)
    nr = tab["theta"].size
    m = np.arange(mmax + 1)
    w = np.where(m == 0, 1.0, 2.0)
    Fb = np.zeros((nr, nder + 1, mmax + 1), dtype=np.complex128)
    for r in range(nr):
        a, n = tab["first"][r], int(tab["nphi"][r])
        ph = np.exp(-1j * m * tab["phi0"][r])
        for (j, k), D in Dbar.items():
            X = np.fft.fft(D[a:a + n])
            Fb[r, j] += w * ph * (-1j * m) ** k * X[m % n]
    return Fb


def _geometry(z, s, phi, a_th, a_ph, th_q, ph_q):
    """theta', phi' (relative to the fixed centre phi_q, wrapped) and beta."""
    n2, u, n, et, d = L.displace(z, s, phi, a_th, a_ph)
    th2 = np.arctan2(np.hypot(n2[:, 0], n2[:, 1]), n2[:, 2])
    ph2 = np.arctan2(n2[:, 1], n2[:, 0])
    beta = np.where(d == 0, 0.0, L.transport_angle(n, u, et, d, th2, ph2))
    return th2 - th_q, L.wrap_pi(ph2 - ph_q), beta


def _jacobian(z, s, phi, a_th, a_ph, th_q, ph_q, h=1e-5):
    """d(dth, dph, beta)/d(a_th, a_ph) by Richardson-extrapolated central differences.

    The step balances the rounding of the differences (~eps/h) against the h^4
    truncation of the extrapolated difference: at h = 1e-5 the error of each row
    is ~1e-10 of its largest entry (a few 1e-7 of the small d(beta)/d(a_th))."""
    out = []
    for comp in (0, 1):
        def D(hh):
            e0 = np.array([hh, 0.0])[comp], np.array([0.0, hh])[comp]
            fp = _geometry(z, s, phi, a_th + e0[0], a_ph + e0[1], th_q, ph_q)
            fm = _geometry(z, s, phi, a_th - e0[0], a_ph - e0[1], th_q, ph_q)
            return [(fp[0] - fm[0]) / (2 * hh), L.wrap_pi(fp[1] - fm[1]) / (2 * hh),
                    L.wrap_pi(fp[2] - fm[2]) / (2 * hh)]
        d1, d2 = D(h), D(h / 2)
        out.append([(4 * b - a) / 3 for a, b in zip(d1, d2)])
    # out[comp][quantity]
    return out


def lens_adjoint(nside: int, lmax: int, order: int, alm_T, alm_E, alm_B, alm_phi, gT, gQ=None, gU=None,
                 rotate: bool = True, nthreads=None):
    tab = hp.ring_table(nside)
    npx = hp.npix(nside)
    pix = np.arange(npx)
    ring, jidx = hp.pix2ring(nside, pix)
    z = tab["z"][ring - 1]
    s = tab["sint"][ring - 1]
    phi = tab["phi0"][ring - 1] + 2.0 * np.pi * jidx / tab["nphi"][ring - 1]
    pol = alm_E is not None
    # ---- forward quantities
    out = L.lens(nside, lmax, order, alm_T, alm_E, alm_B, alm_phi, rotate=rotate, nthreads=nthreads,
                 return_aux=True)
    aux = out["aux"]
    q, dth, dph, beta = aux["q"], aux["dth"], aux["dph"], aux["beta"]
    a_th, a_ph = aux["a_th"], aux["a_ph"]
    maps = L.derivative_maps(nside, lmax, order, alm_T, alm_E, alm_B, nthreads=nthreads)
    th_q, ph_q = hp.pix2ang(nside, q)
    # ---- rotation
    g = {"T": np.asarray(gT, dtype=np.float64)}
    dLdbeta = np.zeros(npx)
    if pol:
        c2, s2 = np.cos(2 * beta), np.sin(2 * beta)
        gQ, gU = np.asarray(gQ, dtype=np.float64), np.asarray(gU, dtype=np.float64)
        g["Q"] = c2 * gQ - s2 * gU
        g["U"] = s2 * gQ + c2 * gU
        if rotate:
            dLdbeta = 2.0 * (gQ * out["U"] - gU * out["Q"])
    # ---- Eq. 4 transpose and dL/dDelta
    pairs = L.derivative_pairs(order)
    Dbar = {f: {} for f in g}
    dLdth = np.zeros(npx)
    dLdph = np.zeros(npx)
    for f in g:
        for (j, k) in pairs:
            wjk = dth ** j * dph ** k / (factorial(j) * factorial(k))
            acc = np.zeros(npx)
            np.add.at(acc, q, wjk * g[f])
            Dbar[f][(j, k)] = acc
            Dq = maps[f][L.map_index(j, k), q]
            if j > 0:
                dLdth += g[f] * Dq * dth ** (j - 1) * dph ** k / (factorial(j - 1) * factorial(k))
            if k > 0:
                dLdph += g[f] * Dq * dth ** j * dph ** (k - 1) / (factorial(j) * factorial(k - 1))
    # ---- coefficient gradients of the unlensed fields
    theta_r = tab["theta"]
    Fb = {f: ring_synthesis_adjoint(Dbar[f], nside, order, lmax) for f in Dbar}
    grads = sht.ring_adjoint(lmax, order, theta_r, Fb["T"], Fb.get("Q"), Fb.get("U"), nthreads=nthreads)
    # ---- deflection
    if alm_phi is not None:
        J = _jacobian(z, s, phi, a_th, a_ph, th_q, ph_q)
        ga_th = dLdth * J[0][0] + dLdph * J[0][1] + dLdbeta * J[0][2]
        ga_ph = dLdth * J[1][0] + dLdph * J[1][1] + dLdbeta * J[1][2]
        Fp = ring_synthesis_adjoint({(1, 0): ga_th, (0, 1): ga_ph / s}, nside, 1, lmax)
        grads["phi"] = sht.ring_adjoint(lmax, 1, theta_r, FbT=Fp, nthreads=nthreads)["T"]
        grads["alpha"] = (ga_th, ga_ph)
    return grads
