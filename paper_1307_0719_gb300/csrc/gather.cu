// Gather + Taylor + rotate: one thread per output pixel (Naess & Louis 2013).
//  1. x = pixel centre, alpha(x) = (a_theta, a_phi) on (e_theta, e_phi)        (Eqs. 1-2)
//  2. x' = end of the geodesic from x along alpha, length |alpha|            (Sec. II.A)
//  3. q = the HEALPix pixel containing x' (ang2pix), x0' = its centre,
//     offsets dth = th' - th_q, dph = ph' - ph_q wrapped to [-pi, pi)         (Sec. II.B)
//  4. s'(x) = sum_{j+k<=n} dth^j dph^k / (j! k!) d_th^j d_ph^k s (x0')        (Eq. 4)
//     for s in {T, Q, U}; the maps are stored pre-divided by j! k! L^(j+k)
//     so the sum is a bivariate polynomial in (L dth, L dph), L = lmax + 1
//  5. Q' + iU' = e^{-2 i beta} (Q + iU), beta the angle at x' of e_theta(x)
//     carried to x' by parallel transport along the geodesic               (Eq. 2, R)
// Pixel geometry and the rotation angle are computed in double precision.
#include <math.h>

#include "legendre.cuh"

namespace tl {

struct PixLoc {
  int ring;  // 0-based ring index
  int idx;   // index within the ring
};

// ring and in-ring index of a RING-scheme pixel
__device__ __forceinline__ PixLoc pix2loc(long long p, int nside, long long npix) {
  const long long ncap = 2LL * nside * (nside - 1);
  PixLoc L;
  if (p < ncap) {
    long long i = (long long)((1.0 + sqrt(1.0 + 2.0 * (double)p)) * 0.5);
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
    long long i = (long long)((1.0 + sqrt(1.0 + 2.0 * (double)q)) * 0.5);
    if (2 * i * (i - 1) > q) --i;
    if (2 * (i + 1) * i <= q) ++i;
    L.ring = (int)(4LL * nside - i) - 1;
    L.idx = (int)(4 * i - 1 - (q - 2 * i * (i - 1)));
  }
  return L;
}

__device__ __forceinline__ long long floordiv2(long long a) { return (a >= 0) ? a / 2 : -((1 - a) / 2); }

// HEALPix ang2pix (RING) from z = cos(theta), s = sin(theta) >= 0 and phi in
// [0, 2pi): belt cells are bounded by the lines N(t + 1/2) -+ (3/4) N z in Z
// (t = 2 phi / pi); cap cells by tp * tmp and (1 - tp) * tmp in Z with
// tmp = N sqrt(3 (1 - |z|)), tp = frac(t) (Gorski et al. 2005).
__device__ __forceinline__ PixLoc ang2loc(double z, double s, double phi, int nside) {
  const double N = (double)nside;
  double t = phi * (2.0 / 3.14159265358979323846);
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
    const double omz = s * s / (1.0 + za);
    const double tmp = N * sqrt(3.0 * omz);
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

template <typename T, int ORDER>
__device__ __forceinline__ T taylor_eval(const T *__restrict__ D, long long stride, long long q, T x, T y) {
  // sum_j x^j sum_k y^k D_{j,k}, map index of (j,k) = (j+k)(j+k+1)/2 + j
  T res = (T)0;
#pragma unroll
  for (int j = ORDER; j >= 0; --j) {
    T inner = (T)0;
#pragma unroll
    for (int k = ORDER - j; k >= 0; --k) {
      const int N = j + k;
      const int mi = N * (N + 1) / 2 + j;
      inner = fma(inner, y, __ldg(D + (long long)mi * stride + q));
    }
    res = fma(res, x, inner);
  }
  return res;
}

template <typename T, int ORDER, bool POL>
__global__ void __launch_bounds__(256) gather_kernel(RingTable rt, int nside, long long npix, double Lnorm,
                                                     const T *__restrict__ a_th, const T *__restrict__ a_ph,
                                                     const T *__restrict__ d3, T *__restrict__ Tout,
                                                     T *__restrict__ Qout, T *__restrict__ Uout, int rotate) {
  constexpr int NM = (ORDER + 1) * (ORDER + 2) / 2;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npix) return;
  const PixLoc loc = pix2loc(p, nside, npix);
  const double z = rt.z[loc.ring], s = rt.sint[loc.ring];
  const double phi = rt.phi0[loc.ring] + 2.0 * 3.14159265358979323846 * (double)loc.idx / (double)rt.nphi[loc.ring];
  const double ath = (double)a_th[p], aph = (double)a_ph[p];
  const double d = hypot(ath, aph);

  long long q = p;
  double dth = 0.0, dph = 0.0, c2b = 1.0, s2b = 0.0;
  if (d > 0.0) {
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
    if (phi2 < 0.0) phi2 += 2.0 * 3.14159265358979323846;
    const double th2 = atan2(s2, nz);
    const PixLoc lq = ang2loc(nz, s2, phi2, nside);
    q = rt.first[lq.ring] + lq.idx;
    const double thq = rt.theta[lq.ring];
    const double phq = rt.phi0[lq.ring] + 2.0 * 3.14159265358979323846 * (double)lq.idx / (double)rt.nphi[lq.ring];
    dth = th2 - thq;
    dph = phi2 - phq;
    if (dph >= 3.14159265358979323846) dph -= 2.0 * 3.14159265358979323846;
    if (dph < -3.14159265358979323846) dph += 2.0 * 3.14159265358979323846;
    if (POL && rotate) {
      // e_theta(x) transported to x' (rotation about n x u by d):
      // t = (1 - cos^2(delta) omc) e_th - sin(delta) cos(delta) omc e_ph - sin(d) cos(delta) n
      const double cdl = ath / d, sdl = aph / d;
      const double sh = sin(0.5 * d);
      const double omc = 2.0 * sh * sh;
      const double ct = 1.0 - cdl * cdl * omc, cph = -sdl * cdl * omc, cn = -sd * cdl;
      const double tx = ct * z * cp + cph * (-sp) + cn * s * cp;
      const double ty = ct * z * sp + cph * cp + cn * s * sp;
      const double tz = ct * (-s) + cn * z;
      // basis at x'
      double cp2 = 1.0, sp2 = 0.0;
      if (s2 > 0.0) {
        cp2 = nx / s2;
        sp2 = ny / s2;
      }
      const double et2x = nz * cp2, et2y = nz * sp2, et2z = -s2;
      const double cb = tx * et2x + ty * et2y + tz * et2z;  // t . e_theta'
      const double sb = -tx * sp2 + ty * cp2;                // t . e_phi'
      const double nrm = cb * cb + sb * sb;
      c2b = (cb * cb - sb * sb) / nrm;
      s2b = 2.0 * cb * sb / nrm;
    }
  }
  const T x = (T)(Lnorm * dth), y = (T)(Lnorm * dph);
  Tout[p] = taylor_eval<T, ORDER>(d3, npix, q, x, y);
  if (POL) {
    const T qv = taylor_eval<T, ORDER>(d3 + (long long)NM * npix, npix, q, x, y);
    const T uv = taylor_eval<T, ORDER>(d3 + 2LL * NM * npix, npix, q, x, y);
    Qout[p] = (T)(c2b * (double)qv + s2b * (double)uv);
    Uout[p] = (T)(-s2b * (double)qv + c2b * (double)uv);
  }
}

template <typename T, int ORDER>
static cudaError_t gather_t(const tl_plan *p, const void *alpha, const void *d3, void *Tq, void *Q, void *U,
                            cudaStream_t s) {
  const int threads = 256;
  const long long blocks = (p->npix + threads - 1) / threads;
  const T *ath = (const T *)alpha;
  const T *aph = ath + p->npix;
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  const int rot = (p->flags & TL_ROTATE) ? 1 : 0;
  // T-only plans keep the T maps at field 0; QU-only plans store Q, U at fields 1, 2
  if (pol)
    gather_kernel<T, ORDER, true><<<(unsigned)blocks, threads, 0, s>>>(
        p->ring, p->nside, p->npix, (double)(p->lmax + 1), ath, aph, (const T *)d3, (T *)Tq, (T *)Q, (T *)U, rot);
  else
    gather_kernel<T, ORDER, false><<<(unsigned)blocks, threads, 0, s>>>(
        p->ring, p->nside, p->npix, (double)(p->lmax + 1), ath, aph, (const T *)d3, (T *)Tq, nullptr, nullptr,
        rot);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t gather_dispatch(const tl_plan *p, const void *a, const void *d3, void *Tq, void *Q, void *U,
                                   cudaStream_t s) {
  switch (p->order) {
    case 0: return gather_t<T, 0>(p, a, d3, Tq, Q, U, s);
    case 1: return gather_t<T, 1>(p, a, d3, Tq, Q, U, s);
    case 2: return gather_t<T, 2>(p, a, d3, Tq, Q, U, s);
    case 3: return gather_t<T, 3>(p, a, d3, Tq, Q, U, s);
    case 4: return gather_t<T, 4>(p, a, d3, Tq, Q, U, s);
    case 5: return gather_t<T, 5>(p, a, d3, Tq, Q, U, s);
    case 6: return gather_t<T, 6>(p, a, d3, Tq, Q, U, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_gather(const tl_plan *p, const void *alpha, const void *d3, void *Tq, void *Q, void *U,
                          cudaStream_t s) {
  return p->precision == TL_FP64 ? gather_dispatch<double>(p, alpha, d3, Tq, Q, U, s)
                                 : gather_dispatch<float>(p, alpha, d3, Tq, Q, U, s);
}

}  // namespace tl
