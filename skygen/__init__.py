"""Seeded synthetic skies: the one module shared by the oracle tests and the GPU path.

It holds no lensing arithmetic. It draws Gaussian spherical-harmonic coefficients
for given power spectra, in the triangular layout idx(l, m) = m(2 lmax + 1 - m)/2 + l
(m >= 0, complex128), and defines the analytic spectra that stand in for the
paper's CAMB LCDM spectra (Sec. II.A).

Random numbers come from a counter-based generator, so any coefficient can be
drawn independently of the others: splitmix64 (Steele, Lea & Flood 2014, the
mixing function published with Java's SplittableRandom) applied to a key built
from (seed, stream, l, m), turned into two uniforms and then into a normal pair by
the Box-Muller transform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "alm_size", "alm_index", "lm_arrays", "splitmix64", "gaussian_pairs",
    "draw_alm", "cl_tt", "cl_ee", "cl_phi", "Workload", "WORKLOADS",
    "make_sky", "batched_lmax_list",
]

ARCMIN = math.pi / (180.0 * 60.0)

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)

# stream ids: one independent Gaussian stream per field
STREAM_T, STREAM_E, STREAM_B, STREAM_PHI = 0, 1, 2, 3


def alm_size(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(lmax: int, l, m):
    return m * (2 * lmax + 1 - m) // 2 + l


def lm_arrays(lmax: int):
    """(l, m) of every entry of the triangular layout, in storage order."""
    ls, ms = [], []
    for m in range(lmax + 1):
        ls.append(np.arange(m, lmax + 1, dtype=np.int64))
        ms.append(np.full(lmax + 1 - m, m, dtype=np.int64))
    return np.concatenate(ls), np.concatenate(ms)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (x + _GOLDEN).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(30))) * _MIX1).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(27))) * _MIX2).astype(np.uint64)
        return z ^ (z >> np.uint64(31))


def _uniform_open(h: np.ndarray) -> np.ndarray:
    """53 random bits -> uniform on the open interval (0, 1)."""
    return ((h >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def gaussian_pairs(seed: int, stream: int, l: np.ndarray, m: np.ndarray):
    """Two independent N(0,1) variates per (l, m), keyed by (seed, stream, l, m)."""
    l = np.asarray(l, dtype=np.uint64)
    m = np.asarray(m, dtype=np.uint64)
    base = splitmix64(np.uint64(seed) * np.uint64(8) + np.uint64(stream))
    key = splitmix64(base ^ ((l << np.uint64(24)) | m))
    h1 = splitmix64(key ^ np.uint64(0x1))
    h2 = splitmix64(key ^ np.uint64(0x2))
    u1, u2 = _uniform_open(h1), _uniform_open(h2)
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


def draw_alm(cl: np.ndarray, lmax: int, seed: int, stream: int) -> np.ndarray:
    """Gaussian coefficients of a real field with spectrum cl[0..lmax].

    a_l0 ~ N(0, C_l) (real); for m > 0, Re and Im ~ N(0, C_l / 2).
    """
    l, m = lm_arrays(lmax)
    g1, g2 = gaussian_pairs(seed, stream, l, m)
    c = np.asarray(cl, dtype=np.float64)[l]
    out = np.empty(l.size, dtype=np.complex128)
    m0 = m == 0
    out.real = np.where(m0, g1 * np.sqrt(c), g1 * np.sqrt(c / 2.0))
    out.imag = np.where(m0, 0.0, g2 * np.sqrt(c / 2.0))
    return out


# ----------------------------------------------------------------------------
# analytic spectra standing in for CAMB (uK^2 for T/E, dimensionless for phi)

def cl_tt(lmax: int, damp: float = 100.0) -> np.ndarray:
    l = np.arange(lmax + 1, dtype=np.float64)
    c = np.zeros(lmax + 1)
    ll = l[2:]
    c[2:] = 1e3 * 2.0 * np.pi / (ll * (ll + 1.0)) * np.exp(-(ll / damp) ** 2)
    return c


def cl_ee(lmax: int, damp_t: float = 100.0, damp_e: float = 800.0) -> np.ndarray:
    l = np.arange(lmax + 1, dtype=np.float64)
    return 0.05 * cl_tt(lmax, damp_t) * np.exp(-(l / damp_e) ** 2)


def cl_phi(lmax: int, rms_arcmin: float = 2.5) -> np.ndarray:
    """C_l^phiphi = A (l+1)^-4 for l >= 1, with A set so that the expected RMS
    deflection sqrt(sum_l (2l+1)/(4 pi) l(l+1) C_l) equals rms_arcmin."""
    l = np.arange(lmax + 1, dtype=np.float64)
    shape = np.zeros(lmax + 1)
    shape[1:] = (l[1:] + 1.0) ** -4
    var = np.sum((2 * l + 1) / (4 * np.pi) * l * (l + 1) * shape)
    target = rms_arcmin * ARCMIN
    return shape * (target ** 2 / var)


@dataclass(frozen=True)
class Workload:
    name: str
    nside: int
    lmax: int
    order: int
    pol: bool
    damp_t: float
    damp_e: float
    seed_t: int
    seed_e: int
    seed_phi: int


WORKLOADS = {
    # Nside 64, lmax 128, order 3, temperature only
    "nside64_lmax128_n3_T": Workload("nside64_lmax128_n3_T", 64, 128, 3, False, 100.0, 800.0, 0, 0, 1),
    # Nside 512, lmax 1024, order 4, T+Q/U
    "nside512_lmax1024_n4_TQU": Workload("nside512_lmax1024_n4_TQU", 512, 1024, 4, True, 100.0, 800.0, 2, 3, 4),
    # Nside 2048, lmax 4096, order 4 (2..6 swept), T+Q/U, damping scales x4
    "nside2048_lmax4096_n4_TQU": Workload("nside2048_lmax4096_n4_TQU", 2048, 4096, 4, True, 400.0, 3200.0, 2, 3, 4),
    # Nside 2048, lmax 4096, order 4, temperature only: the full-size ring FFT and gather
    # kernels in a few GB (profiling)
    "nside2048_lmax4096_n4_T": Workload("nside2048_lmax4096_n4_T", 2048, 4096, 4, False, 400.0, 3200.0, 2, 3, 4),
    # Nside 1024, lmax 2048, order 4: differentiation workload (targets from seed 9000)
    "nside1024_lmax2048_n4_TQU": Workload("nside1024_lmax2048_n4_TQU", 1024, 2048, 4, True, 400.0, 3200.0, 2, 3, 4),
}


def make_sky(nside: int, lmax: int, pol: bool, seed_t: int, seed_e: int, seed_phi: int,
             damp_t: float = 100.0, damp_e: float = 800.0, rms_arcmin: float = 2.5,
             b_scale: float = 0.0):
    """Unlensed T (and E, B) coefficients plus the lensing potential's.

    B is zero unless b_scale > 0 (then C_l^BB = b_scale * C_l^EE, drawn from
    its own stream of seed_e), which tests use to exercise the B path.
    Returns a dict of complex128 arrays in the triangular layout.
    """
    out = {"T": draw_alm(cl_tt(lmax, damp_t), lmax, seed_t, STREAM_T)}
    if pol:
        ee = cl_ee(lmax, damp_t, damp_e)
        out["E"] = draw_alm(ee, lmax, seed_e, STREAM_E)
        if b_scale > 0.0:
            out["B"] = draw_alm(b_scale * ee, lmax, seed_e, STREAM_B)
        else:
            out["B"] = np.zeros(alm_size(lmax), dtype=np.complex128)
    out["phi"] = draw_alm(cl_phi(lmax, rms_arcmin), lmax, seed_phi, STREAM_PHI)
    return out


def workload_sky(name: str):
    w = WORKLOADS[name]
    return make_sky(w.nside, w.lmax, w.pol, w.seed_t, w.seed_e, w.seed_phi, w.damp_t, w.damp_e)


def batched_lmax_list(n: int = 64, first_seed: int = 100):
    """Uneven batch: realization i uses seed first_seed+i; its lmax is drawn
    uniformly from {512, 1024, 2048, 3000} by the first splitmix64 output of
    that seed, and its Nside is the next power of two >= lmax/2."""
    choices = (512, 1024, 2048, 3000)
    out = []
    for i in range(n):
        s = first_seed + i
        u = int(splitmix64(np.array([s], dtype=np.uint64))[0])
        lmax = choices[u % 4]
        nside = 1
        while nside < lmax / 2:
            nside *= 2
        out.append((s, nside, lmax))
    return out
