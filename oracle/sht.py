"""ctypes wrapper over the oracle's C core (test infrastructure only).

See sht.c for the definitions (spin-weighted lambda recurrence, ladder-identity
theta derivatives, HEALPix polarisation convention)."""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _threads() -> int:
    env = os.environ.get("ORACLE_THREADS")
    if env:
        return int(env)
    return os.cpu_count() or 1


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_spin_lambda.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
        L.orc_spin_lambda_derivs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, dp]
        L.orc_ring_coeffs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.orc_point_sum.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                    ctypes.c_int, dp, ctypes.c_int]
        L.orc_ring_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vp(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def spin_lambda(lmax: int, m: int, s: int, theta: float) -> np.ndarray:
    out = np.zeros(lmax + 1)
    lib().orc_spin_lambda(lmax, m, s, float(theta), _p(out))
    return out


def spin_lambda_derivs(lmax: int, m: int, s: int, nder: int, theta: float) -> np.ndarray:
    """[nder+1, lmax+1]: d^j/dtheta^j slambda_lm(theta)."""
    out = np.zeros((nder + 1, lmax + 1))
    lib().orc_spin_lambda_derivs(lmax, m, s, nder, float(theta), _p(out))
    return out


def _as_ri(alm):
    if alm is None:
        return None
    a = np.ascontiguousarray(np.asarray(alm, dtype=np.complex128))
    return a.view(np.float64)


def ring_coeffs(lmax: int, nder: int, theta, alm_T=None, alm_E=None, alm_B=None,
                mmax: int | None = None, nthreads: int | None = None):
    """Fourier coefficients F^{s,j}_m(theta_r) of the theta-derivatives, for s in
    {T, Q, U}. Returns dict of complex128 arrays [nth, nder+1, mmax+1]."""
    theta = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).ravel())
    mmax = lmax if mmax is None else mmax
    nth = theta.size
    shape = (nth, nder + 1, mmax + 1)
    out = {}
    FT = np.zeros(shape, dtype=np.complex128) if alm_T is not None else None
    pol = alm_E is not None or alm_B is not None
    FQ = np.zeros(shape, dtype=np.complex128) if pol else None
    FU = np.zeros(shape, dtype=np.complex128) if pol else None
    aT, aE, aB = _as_ri(alm_T), _as_ri(alm_E), _as_ri(alm_B)
    lib().orc_ring_coeffs(lmax, mmax, nder, nth, _p(theta), _vp(aT), _vp(aE), _vp(aB),
                          _vp(FT), _vp(FQ), _vp(FU), nthreads or _threads())
    if FT is not None:
        out["T"] = FT
    if pol:
        out["Q"], out["U"] = FQ, FU
    return out


def point_sum(F: np.ndarray, phi, j: int, k: int, nthreads: int | None = None) -> np.ndarray:
    """Direct Fourier sum Re[F_0 + 2 sum_m (i m)^k F^j_m e^{i m phi}] per point."""
    F = np.ascontiguousarray(F, dtype=np.complex128)
    npts, nd1, m1 = F.shape
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).ravel())
    out = np.zeros(npts)
    lib().orc_point_sum(m1 - 1, nd1 - 1, npts, _p(F.view(np.float64)), _p(phi), j, k, _p(out),
                        nthreads or _threads())
    return out


def ring_adjoint(lmax: int, nder: int, theta, FbT=None, FbQ=None, FbU=None, nthreads: int | None = None):
    """Transpose of ring_coeffs: coefficient gradients (dL/dRe + i dL/dIm) from the
    per-ring gradients Fb[r, j, m] (complex). Returns dict with keys among T, E, B."""
    theta = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).ravel())
    any_f = FbT if FbT is not None else FbQ
    nth, nd1, m1 = any_f.shape
    na = (lmax + 1) * (lmax + 2) // 2
    out = {}
    aT = np.zeros(na, dtype=np.complex128) if FbT is not None else None
    aE = np.zeros(na, dtype=np.complex128) if FbQ is not None else None
    aB = np.zeros(na, dtype=np.complex128) if FbQ is not None else None
    c = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.complex128)
    fT, fQ, fU = c(FbT), c(FbQ), c(FbU)
    lib().orc_ring_adjoint(lmax, m1 - 1, nd1 - 1, nth, _p(theta), _vp(None if fT is None else fT.view(np.float64)),
                           _vp(None if fQ is None else fQ.view(np.float64)),
                           _vp(None if fU is None else fU.view(np.float64)),
                           _vp(None if aT is None else aT.view(np.float64)),
                           _vp(None if aE is None else aE.view(np.float64)),
                           _vp(None if aB is None else aB.view(np.float64)), nthreads or _threads())
    if aT is not None:
        out["T"] = aT
    if aE is not None:
        out["E"], out["B"] = aE, aB
    return out
