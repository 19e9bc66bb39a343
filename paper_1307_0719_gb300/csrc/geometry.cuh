// HEALPix RING pixel geometry on the device (Gorski et al. 2005) and the
// double-precision displacement geometry of the lensing gather (Naess & Louis
// 2013, Secs. II.A-II.B; rotation R of Eq. 2), shared by the gather and its adjoint.
#pragma once

#include <math.h>

#include "legendre.cuh"

namespace tl {

static constexpr double kPiD = 3.14159265358979323846;

struct PixLoc {
  int ring;  // 0-based ring index
  int idx;   // index within the ring
};

// ring and in-ring index of a RING-scheme pixel (the ring from a float square-root
// estimate, off by at most one, then corrected in integers)
__device__ __forceinline__ PixLoc pix2loc(long long p, int nside, long long npix) {
  const long long ncap = 2LL * nside * (nside - 1);
  PixLoc L;
  if (p < ncap) {
    long long i = (long long)((1.0f + sqrtf(1.0f + 2.0f * (float)p)) * 0.5f);
    if (2 * i * (i - 1) > p) --i;
    if (2 * (i + 1) * i <= p) ++i;
    L.ring = (int)i - 1;
    L.idx = (int)(p - 2 * i * (i - 1));
  } else if (p < npix - ncap) {
    long long q = p - ncap;
    long long i = q / (4LL * nside) + nside;
    L.ring = (int)i - 1;
    L.idx = (int)(q - (i - nside) * 4LL * nside);
  } else {
    long long q = npix - 1 - p;
    long long i = (long long)((1.0f + sqrtf(1.0f + 2.0f * (float)q)) * 0.5f);
    if (2 * i * (i - 1) > q) --i;
    if (2 * (i + 1) * i <= q) ++i;
    L.ring = (int)(4LL * nside - i) - 1;
    L.idx = (int)(4 * i - 1 - (q - 2 * i * (i - 1)));
  }
  return L;
}

__device__ __forceinline__ long long floordiv2(long long a) { return (a >= 0) ? a / 2 : -((1 - a) / 2); }

// HEALPix ang2pix (RING) from z = cos(theta), omz = 1 - |z| and phi in [0, 2pi):
// belt cells are bounded by the lines N(t + 1/2) -+ (3/4) N z in Z (t = 2 phi / pi);
// cap cells by tp * tmp and (1 - tp) * tmp in Z with tmp = N sqrt(3 (1 - |z|)),
// tp = frac(t) (Gorski et al. 2005).
__device__ __forceinline__ PixLoc ang2loc(double z, double omz, double phi, int nside) {
  const double N = (double)nside;
  double t = phi * (2.0 / kPiD);
  if (t >= 4.0) t -= 4.0;
  if (t < 0.0) t += 4.0;
  const double za = fabs(z);
  PixLoc L;
  if (za <= 2.0 / 3.0) {
    const double a = N * (0.5 + t), b = 0.75 * N * z;
    const long long jp = (long long)floor(a - b);
    const long long jm = (long long)floor(a + b);
    long long ir = nside + 1 + jp - jm;  // 1 .. 2N+1
    if (ir < 1) ir = 1;                   // rounding exactly at |z| = 2/3
    if (ir > 2LL * nside + 1) ir = 2LL * nside + 1;
    const long long kshift = 1 - (ir & 1);
    long long ip = floordiv2(jp + jm - nside + kshift + 1);
    const long long n4 = 4LL * nside;
    ip %= n4;
    if (ip < 0) ip += n4;
    L.ring = (int)(nside - 2 + ir);
    L.idx = (int)ip;
  } else {
    const double tp = t - floor(t);
    const double tmp = N * sqrt(3.0 * (omz > 0.0 ? omz : 0.0));
    long long jp = (long long)floor(tp * tmp);
    long long jm = (long long)floor((1.0 - tp) * tmp);
    long long ir = jp + jm + 1;
    if (ir > nside) ir = nside;  // guards rounding exactly at |z| = 2/3
    long long ip = (long long)floor(t * (double)ir);
    ip %= 4 * ir;
    if (ip < 0) ip += 4 * ir;
    L.ring = (z > 0.0) ? (int)ir - 1 : (int)(4LL * nside - ir) - 1;
    L.idx = (int)ip;
  }
  return L;
}

// ang2loc in single precision, for the float gather. z, omz = 1 - |z| and
// t = 2 phi / pi come rounded to float (|z| <= 1, t in [0, 4)), so every floor
// argument below carries an absolute error under N * 1e-6 (input rounding of t,
// z and omz times at most 4N, plus the products' own rounding). When one lies
// within eps = N * 2.5e-6 of an integer, or |z| within 1e-6 of 2/3, or t within
// 1e-6 of an integer, `ok` is false and the caller takes ang2loc in double;
// otherwise both make the same decisions, so the cell is ang2loc's.
__device__ __forceinline__ PixLoc ang2loc_f(float z, float omz, float t, int nside, bool &ok) {
  const float N = (float)nside, eps = N * 2.5e-6f;
  if (t >= 4.0f) t -= 4.0f;
  if (t < 0.0f) t += 4.0f;
  const float za = fabsf(z);
  ok = fabsf(za - (2.0f / 3.0f)) >= 1e-6f;
  PixLoc L;
  if (za <= 2.0f / 3.0f) {
    const float a = N * (0.5f + t), b = 0.75f * N * z;
    const float x1 = a - b, x2 = a + b;
    ok = ok && fabsf(x1 - rintf(x1)) >= eps && fabsf(x2 - rintf(x2)) >= eps;
    const int jp = (int)floorf(x1), jm = (int)floorf(x2);
    int ir = nside + 1 + jp - jm;
    if (ir < 1) ir = 1;
    if (ir > 2 * nside + 1) ir = 2 * nside + 1;
    const int kshift = 1 - (ir & 1);
    const int v = jp + jm - nside + kshift + 1;
    int ip = (v >= 0) ? v / 2 : -((1 - v) / 2);
    const int n4 = 4 * nside;
    ip %= n4;
    if (ip < 0) ip += n4;
    L.ring = nside - 2 + ir;
    L.idx = ip;
  } else {
    ok = ok && fabsf(t - rintf(t)) >= 1e-6f;
    const float tp = t - floorf(t);
    const float tmp = N * sqrtf(3.0f * (omz > 0.0f ? omz : 0.0f));
    const float x1 = tp * tmp, x2 = (1.0f - tp) * tmp;
    ok = ok && fabsf(x1 - rintf(x1)) >= eps && fabsf(x2 - rintf(x2)) >= eps;
    const int jp = (int)floorf(x1), jm = (int)floorf(x2);
    int ir = jp + jm + 1;
    if (ir > nside) ir = nside;
    const float x3 = t * (float)ir;
    ok = ok && fabsf(x3 - rintf(x3)) >= eps;
    int ip = (int)floorf(x3);
    ip %= 4 * ir;
    if (ip < 0) ip += 4 * ir;
    L.ring = (z > 0.0f) ? ir - 1 : 4 * nside - ir - 1;
    L.idx = ip;
  }
  return L;
}

// Pixel lookup of x' in increments from the output pixel p = (ring, idx), for the
// float gather. In HEALPix's cell coordinates every pixel centre sits at
// half-integers: in the belt x1 = N(t + 1/2) - (3/4) N z = idx + (sh + i - N)/2 and
// x2 = N(t + 1/2) + (3/4) N z = idx + (3N + sh - i)/2 (i = ring + 1, sh the ring's
// half-pixel shift); in a cap, with i the ring's distance from its pole,
// tmp = N sqrt(3 (1 - |z|)) = i and t = f + (k + 1/2)/i (face f, k = idx - f i), so
// x1 = tp tmp = k + 1/2 and x2 = (1 - tp) tmp = i - k - 1/2. The displaced
// coordinates are then an exact integer plus 1/2 plus a term e formed from
// dz = z' - z and dt = t' - t alone, whose rounding error is relative to the
// displacement terms rather than to the absolute position. dz and dt carry
// errors under a few units in the last place relative to dzmag (the sum of the
// magnitudes of the terms dz was formed from) and |dt|; every floor below is
// certified against kIncRel times the magnitude of its terms plus 1e-6.
// Returns 1 with the cell in L, 0 when a decision is within its bound (the caller
// defers the pixel to the double pass), 2 when x' certainly lies in another
// region (belt / cap) than p (the caller then takes ang2loc_f).
constexpr float kIncRel = 4e-6f;
__device__ __forceinline__ int ang2loc_inc(int nside, int ring, int idx, int sh, float dz, float dzmag, float dt,
                                           PixLoc &L) {
  const int N = nside, i = ring + 1;
  const float Nf = (float)N;
  if (i >= N && i <= 3 * N) {  // belt pixel
    const float a = Nf * dt, b = 0.75f * Nf * dz, bm = 0.75f * Nf * dzmag;
    // |z'| <= 2/3  <=>  (i - 3N)/2 <= b <= (i - N)/2, both bounds exact
    const float lo = 0.5f * (float)(i - 3 * N), hi = 0.5f * (float)(i - N);
    const float eb = 1e-6f + kIncRel * bm;
    if (fabsf(b - lo) < eb || fabsf(b - hi) < eb) return 0;
    if (b < lo || b > hi) return 2;
    const float e = 1e-6f + kIncRel * (fabsf(a) + bm);
    const float f1 = 0.5f + (a - b), f2 = 0.5f + (a + b);
    if (fabsf(f1 - rintf(f1)) < e || fabsf(f2 - rintf(f2)) < e) return 0;
    const int jp = idx + ((sh + i - N - 1) >> 1) + (int)floorf(f1);
    const int jm = idx + ((3 * N + sh - i - 1) >> 1) + (int)floorf(f2);
    int ir = N + 1 + jp - jm;  // 1 .. 2N+1 by the region test
    if (ir < 1) ir = 1;
    if (ir > 2 * N + 1) ir = 2 * N + 1;
    const int v = jp + jm - N + (1 - (ir & 1)) + 1;
    int ip = (v >= 0) ? v / 2 : -((1 - v) / 2);
    ip %= 4 * N;
    if (ip < 0) ip += 4 * N;
    L.ring = N - 2 + ir;
    L.idx = ip;
    return 1;
  }
  const bool north = i < N;
  const int ir = north ? i : 4 * N - i;  // p's ring counted from its pole
  const float irf = (float)ir;
  // tmp'^2 - ir^2 = 3 N^2 ((1 - |z'|) - (1 - |z|))
  const float c = 3.0f * Nf * Nf * (north ? -dz : dz), cm = 3.0f * Nf * Nf * dzmag;
  const float s2 = irf * irf + c;
  if (!(s2 > 0.0f)) return 0;
  const float den = sqrtf(s2) + irf;
  const float del = c / den, delm = cm / den;  // tmp' - ir, no cancellation
  // x' in the same cap  <=>  tmp' < N
  const float gap = (float)(N - ir);
  if (fabsf(del - gap) < 1e-6f + kIncRel * delm) return 0;
  if (del > gap) return 2;
  const int f = idx / ir, k = idx - f * ir;
  const float v = ((float)k + 0.5f) / irf + dt;  // t' - f
  if (fabsf(v - rintf(v)) < 1e-6f + kIncRel * fabsf(dt)) return 0;
  const int fl = (int)floorf(v);
  const float tp = v - (float)fl;  // frac(t')
  const float a = dt * irf;
  const float g1 = 0.5f + (a + tp * del), g2 = 0.5f + ((1.0f - tp) * del - a);
  const float e = 1e-6f + kIncRel * (fabsf(a) + delm);
  if (fabsf(g1 - rintf(g1)) < e || fabsf(g2 - rintf(g2)) < e) return 0;
  const int K1 = k - fl * ir;
  const int jp = K1 + (int)floorf(g1);
  const int jm = ir - 1 - K1 + (int)floorf(g2);
  int ir2 = jp + jm + 1;  // 1 .. N by the region test
  if (ir2 < 1) ir2 = 1;
  if (ir2 > N) ir2 = N;
  // ip = floor(t' ir2) with t' ir2 = f ir2 + (2k + 1) ir2 / (2 ir) + dt ir2
  const int num = (2 * k + 1) * ir2, twoir = 2 * ir;
  const int qq = num / twoir;
  const float g3 = (float)(num - qq * twoir) / (float)twoir + dt * (float)ir2;
  if (fabsf(g3 - rintf(g3)) < 1e-6f + kIncRel * fabsf(dt) * (float)ir2) return 0;
  int ip = f * ir2 + qq + (int)floorf(g3);
  ip %= 4 * ir2;
  if (ip < 0) ip += 4 * ir2;
  L.ring = north ? ir2 - 1 : 4 * N - ir2 - 1;
  L.idx = ip;
  return 1;
}

__device__ __forceinline__ double ring_phi(const RingTable &rt, int ring, int idx) {
  return fma((double)idx, rt.dphi[ring], rt.phi0[ring]);
}

struct Geo {
  long long q;
  double dth, dph;  // offsets to the expansion centre
  double c2b, s2b;  // cos 2 beta, sin 2 beta
};

// Gather geometry options (plan flags): x' by naive coordinate addition instead of
// the geodesic; expansion about the output pixel itself instead of the cell
// containing x'. The rotation R keeps the geodesic transport angle either way.
constexpr int kGeoNaive = 2, kGeoAtPixel = 4;

// Double-precision geometry (any pixel, any deflection). p: the output pixel, at
// (theta, phi) with z = cos theta, s = sin theta; mode: kGeoNaive | kGeoAtPixel bits.
__device__ __forceinline__ void geo64(const RingTable &rt, int nside, long long p, double theta, double z, double s,
                                      double phi, double ath, double aph, bool rot, int mode, Geo &g) {
  const double d = hypot(ath, aph);
  double sp, cp;
  sincos(phi, &sp, &cp);
  double sd, cd;
  sincos(d, &sd, &cd);
  const double sinc = sd / d;
  // n = (s cp, s sp, z), e_th = (z cp, z sp, -s), e_ph = (-sp, cp, 0)
  const double ux = ath * z * cp - aph * sp, uy = ath * z * sp + aph * cp, uz = -ath * s;
  const double nx = cd * s * cp + sinc * ux;
  const double ny = cd * s * sp + sinc * uy;
  const double nz = cd * z + sinc * uz;
  const double s2 = hypot(nx, ny);
  double phi2 = atan2(ny, nx);
  if (phi2 < 0.0) phi2 += 2.0 * kPiD;
  double th2 = atan2(s2, nz);
  double z2 = nz, omz2 = s2 * s2 / (1.0 + fabs(nz));  // 1 - |z'| without cancellation
  if (mode & kGeoNaive) {
    // theta' = theta + a_theta, phi' = phi + a_phi / sin theta; past a pole the point
    // continues on the other side (theta' -> -theta' or 2 pi - theta', phi' + pi)
    th2 = theta + ath;
    phi2 = phi + aph / s;
    if (th2 < 0.0) {
      th2 = -th2;
      phi2 += kPiD;
    } else if (th2 > kPiD) {
      th2 = 2.0 * kPiD - th2;
      phi2 += kPiD;
    }
    phi2 = fmod(phi2, 2.0 * kPiD);
    if (phi2 < 0.0) phi2 += 2.0 * kPiD;
    double sn, cn;
    sincos(th2, &sn, &cn);
    z2 = cn;
    omz2 = sn * sn / (1.0 + fabs(cn));
  }
  double dph;
  if (mode & kGeoAtPixel) {
    g.q = p;
    g.dth = th2 - theta;
    dph = phi2 - phi;
  } else {
    const PixLoc lq = ang2loc(z2, omz2, phi2, nside);
    g.q = rt.first[lq.ring] + lq.idx;
    g.dth = th2 - rt.theta[lq.ring];
    dph = phi2 - ring_phi(rt, lq.ring, lq.idx);
  }
  if (dph >= kPiD) dph -= 2.0 * kPiD;
  if (dph < -kPiD) dph += 2.0 * kPiD;
  g.dph = dph;
  g.c2b = 1.0;
  g.s2b = 0.0;
  if (rot) {
    // e_theta(x) transported to x' (rotation about n x u by d):
    // t = (1 - cos^2(delta) omc) e_th - sin(delta) cos(delta) omc e_ph - sin(d) cos(delta) n
    const double cdl = ath / d, sdl = aph / d;
    const double sh = sin(0.5 * d);
    const double omc = 2.0 * sh * sh;
    const double ct = 1.0 - cdl * cdl * omc, cph = -sdl * cdl * omc, cn = -sd * cdl;
    const double tx = ct * z * cp + cph * (-sp) + cn * s * cp;
    const double ty = ct * z * sp + cph * cp + cn * s * sp;
    const double tz = ct * (-s) + cn * z;
    double cp2 = 1.0, sp2 = 0.0;
    if (s2 > 0.0) {
      cp2 = nx / s2;
      sp2 = ny / s2;
    }
    const double cb = tx * nz * cp2 + ty * nz * sp2 - tz * s2;  // t . e_theta'
    const double sb = -tx * sp2 + ty * cp2;                      // t . e_phi'
    const double nrm = cb * cb + sb * sb;
    g.c2b = (cb * cb - sb * sb) / nrm;
    g.s2b = 2.0 * cb * sb / nrm;
  }
}

}  // namespace tl
