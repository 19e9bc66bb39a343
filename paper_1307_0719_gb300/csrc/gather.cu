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
//
// Geometry. The double-precision form evaluates x' as a unit vector and takes
// atan2 of its components. The mixed form (float maps) works in increments: in a
// frame turned to the pixel's longitude, the displaced point is
//     X = s cos d + z a_th sinc d,  Y = a_ph sinc d,  Z - z = -z (1 - cos d) - s a_th sinc d,
// and  phi' - phi_p = atan2(Y, X),
//      th' - th_p   = atan2(a_th sinc d + z w, cos d + s w),  w = Y^2 / (rho + X),  rho = |(X, Y)|,
// which carry no cancellation, so float arithmetic gives them to ~1e-7 relative.
// The pixel lookup runs in single precision with a certified error bound: every
// floor whose argument lies within the bound of an integer marks the pixel as
// uncertain. It works in increments from the output pixel, whose centre sits at
// half-integer cell coordinates, so the bound scales with the displacement rather
// than with the position (ang2loc_inc); only a point that crosses between belt and
// cap takes the whole-coordinate lookup (ang2loc_f, bound N * 2.5e-6 cells). The
// offsets to the expansion centre subtract centre differences taken from exact
// integers and hi/lo float ring colatitudes. Pixels deflected by more than
// sin(theta)/4 (near a pole, where rho + X could cancel for a point carried over
// it) or by more than 0.02 rad, and pixels whose float lookup is uncertain, are
// not computed in the float kernel: it appends them to a queue (one global atomic
// per block) and a second kernel runs them with the double geometry, so that no
// warp of the float kernel waits on the FP64 pipe.
#include <math.h>

#include "geometry.cuh"

namespace tl {

// Increment-form geometry in float (see the header comment), pixel lookup in float.
// Returns false when the lookup cannot certify the cell (the caller then defers the
// pixel to the double pass); else the expansion pixel q and, in float, the scaled
// offsets x = L dth, y = L dph and cos 2 beta, sin 2 beta.
struct Geo32 {
  long long q;
  float x, y, c2b, s2b;
};
// The pixel is (ring, idx), fr its float ring record (z, sin theta, 1 - |z|, theta
// hi, theta lo). No double arithmetic.
__device__ __forceinline__ bool geo32(const RingTable &rt, int nside, long long p, int ring, int idx, float4 fr,
                                      float th_lo, float ath, float aph, bool rot, int mode, float Lf, Geo32 &g) {
  const float d2 = ath * ath + aph * aph;
  const float d = sqrtf(d2);
  float sh, ch;
  sincosf(0.5f * d, &sh, &ch);
  const float hsinc = (d > 0.0f) ? sh / (0.5f * d) : 1.0f;  // sinc(d/2)
  const float sinc = hsinc * ch;                             // sin(d)/d
  const float omc = 2.0f * sh * sh;                          // 1 - cos d
  const float zf = fr.x, sf = fr.y;
  const float X = sf * (1.0f - omc) + zf * ath * sinc;
  const float Y = aph * sinc;
  const float dz = -zf * omc - sf * ath * sinc;
  const float rho = sqrtf(X * X + Y * Y);
  const float w = Y * Y / (rho + X);
  float dthp = atan2f(ath * sinc + zf * w, (1.0f - omc) + sf * w);  // th' - th_p
  float dphp = atan2f(Y, X);                                        // phi' - phi_p
  float dzx = dz;                                                   // z' - z_p
  float dzmag = fabsf(zf * omc) + fabsf(sf * ath * sinc);           // its terms' sizes
  if (mode & kGeoNaive) {
    // naive addition: th' - th_p = a_th, phi' - phi_p = a_ph / sin th; points that
    // could be carried past a pole (|alpha| > sin th / 4) take the double pass
    float sa, ca;
    sincosf(0.5f * ath, &sa, &ca);
    dthp = ath;
    dphp = aph * __ldg(rt.rsinf + ring);
    dzx = -sf * (2.0f * sa * ca) - zf * (2.0f * sa * sa);  // cos(th + a) - cos th
    dzmag = fabsf(sf * (2.0f * sa * ca)) + fabsf(zf * (2.0f * sa * sa));
  }
  const int np = rt.nphi[ring];
  const int shp = __double_as_longlong(rt.phi0[ring]) != 0;  // phi0 >= 0: an integer test
  g.c2b = 1.0f;
  g.s2b = 0.0f;
  if (rot) {
    // t = (1 - a_th^2 h) e_th - a_ph a_th h e_ph - a_th sinc n, h = (1 - cos d)/d^2,
    // in the frame turned to phi_p: e_th = (z, 0, -s), e_ph = (0, 1, 0), n = (s, 0, z);
    // read at the geodesic end point (X, Y, Z)
    const float h = 0.5f * hsinc * hsinc;
    const float ct = 1.0f - ath * ath * h;
    const float tx = ct * zf - ath * sinc * sf;
    const float ty = -aph * ath * h;
    const float tz = -ct * sf - ath * sinc * zf;
    const float Z = zf + dz;
    const float cb = Z * (tx * X + ty * Y) / rho - tz * rho;  // t . e_theta'
    const float sb = (-tx * Y + ty * X) / rho;                // t . e_phi'
    const float nrm = cb * cb + sb * sb;
    g.c2b = (cb * cb - sb * sb) / nrm;
    g.s2b = 2.0f * cb * sb / nrm;
  }
  if (mode & kGeoAtPixel) {  // expansion about the output pixel itself
    g.q = p;
    g.x = Lf * dthp;
    float dph = dphp;
    if (dph >= (float)kPiD) dph -= 2.0f * (float)kPiD;
    if (dph < -(float)kPiD) dph += 2.0f * (float)kPiD;
    g.y = Lf * dph;
    return true;
  }
  // pixel lookup in float where every decision clears its error bound: in
  // increments from p (ang2loc_inc), or, for x' in the other region (belt / cap),
  // from the whole coordinates (ang2loc_f); else the pixel goes to the double pass.
  // Pixel centres: phi = 2 pi (idx + sh/2) / nphi, sh = 1 on half-pixel-shifted rings.
  const float dt = dphp * (float)(2.0 / kPiD);  // t' - t_p, t = 2 phi / pi
  PixLoc lq;
  const int how = ang2loc_inc(nside, ring, idx, shp, dzx, dzmag, dt, lq);
  if (how == 0) return false;
  if (how == 2) {
    const float tf = (float)(4 * idx + 2 * shp) / (float)np + dt;
    bool ok;
    lq = ang2loc_f(zf + dzx, fr.z - (zf >= 0.0f ? dzx : -dzx), tf, nside, ok);
    if (!ok) return false;
  }
  g.q = rt.first[lq.ring] + lq.idx;
  // theta_q - theta_p from the hi/lo parts: the hi difference is exact (nearby
  // rings, Sterbenz), so this is the double difference rounded once
  const float4 fq = __ldg((const float4 *)(rt.ringf + 8 * (size_t)lq.ring));
  const float thq_lo = __ldg(rt.ringf + 8 * (size_t)lq.ring + 4);
  g.x = Lf * (dthp - ((fq.w - fr.w) + (thq_lo - th_lo)));
  // centre offset phi_q - phi_p = 2 pi [(2 idx_q + sh_q) nphi_p - (2 idx_p + sh_p) nphi_q] / (2 nphi_q nphi_p),
  // the numerator an exact integer, wrapped to [-pi, pi) exactly
  const int nq = rt.nphi[lq.ring];
  const int shq = __double_as_longlong(rt.phi0[lq.ring]) != 0;
  const long long den = 2LL * nq * np;
  long long num = (long long)(2 * lq.idx + shq) * np - (long long)(2 * idx + shp) * nq;
  num %= den;
  if (num >= den / 2) num -= den;
  if (num < -den / 2) num += den;
  const float dc = (float)num * ((float)(2.0 * kPiD) / (float)den);
  float dph = dphp - dc;
  if (dph >= (float)kPiD) dph -= 2.0f * (float)kPiD;
  if (dph < -(float)kPiD) dph += 2.0f * (float)kPiD;
  g.y = Lf * dph;
  return true;
}

// sum_j x^j sum_k y^k D_{j,k} at the expansion pixel, map index of (j,k) =
// (j+k)(j+k+1)/2 + j; D: the field's first map in the tiled layout, qoff the pixel's
// element (d3_pix)
template <typename T, int ORDER>
__device__ __forceinline__ T taylor_eval(const T *__restrict__ D, long long qoff, T x, T y) {
  T res = (T)0;
#pragma unroll
  for (int j = ORDER; j >= 0; --j) {
    T inner = (T)0;
#pragma unroll
    for (int k = ORDER - j; k >= 0; --k) {
      const int N = j + k;
      const int mi = N * (N + 1) / 2 + j;
      inner = fma(inner, y, __ldg(D + qoff + (long long)mi * kD3Tile));
    }
    res = fma(res, x, inner);
  }
  return res;
}

// Eq. 4 at the expansion pixel q and the rotation, stored for output pixel p; d3 in
// the pixel-tiled layout (tile: elements between tiles).
template <typename T, int ORDER, bool POL>
__device__ __forceinline__ void taylor_store(long long tile, long long p, long long q, T x, T y, T c2, T s2,
                                             const T *__restrict__ d3, T *__restrict__ Tout, T *__restrict__ Qout,
                                             T *__restrict__ Uout) {
  constexpr int NM = (ORDER + 1) * (ORDER + 2) / 2;
  const long long qoff = d3_pix(q, tile);
  Tout[p] = taylor_eval<T, ORDER>(d3, qoff, x, y);
  if (POL) {
    const T qv = taylor_eval<T, ORDER>(d3 + NM * kD3Tile, qoff, x, y);
    const T uv = taylor_eval<T, ORDER>(d3 + 2 * NM * kD3Tile, qoff, x, y);
    Qout[p] = c2 * qv + s2 * uv;
    Uout[p] = -s2 * qv + c2 * uv;
  }
}

// One thread per output pixel. The double form computes every pixel; the float
// form defers the pixels that need the double geometry (see the header comment)
// to queue[0 .. *qcount), filled with one global atomic per block.
template <typename T, int ORDER, bool POL>
__global__ void __launch_bounds__(256) gather_kernel(RingTable rt, int nside, long long npix, double Lnorm,
                                                     const T *__restrict__ a_th, const T *__restrict__ a_ph,
                                                     const T *__restrict__ d3, T *__restrict__ Tout,
                                                     T *__restrict__ Qout, T *__restrict__ Uout, int rotate,
                                                     int *__restrict__ queue, int *__restrict__ qcount,
                                                     long long tile, int mode) {
  constexpr bool FAST = sizeof(T) == 4;
  __shared__ int s_cnt, s_base;
  __shared__ int s_list[FAST ? 256 : 1];
  if (FAST) {
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
  }
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool rot = POL && rotate;
  bool defer = false;
  if (p < npix) {
    const PixLoc loc = pix2loc(p, nside, npix);
    const T ath = a_th[p], aph = a_ph[p];
    long long q = p;
    T x = (T)0, y = (T)0, c2 = (T)1, s2 = (T)0;
    if (ath != (T)0 || aph != (T)0) {
      if (FAST) {
        const float4 fr = __ldg((const float4 *)(rt.ringf + 8 * (size_t)loc.ring));
        Geo32 g;
        const float d2 = (float)(ath * ath + aph * aph);
        defer = !(d2 < 4e-4f && d2 < 0.0625f * fr.y * fr.y) ||
                !geo32(rt, nside, p, loc.ring, loc.idx, fr, __ldg(rt.ringf + 8 * (size_t)loc.ring + 4), (float)ath,
                       (float)aph, rot, mode, (float)Lnorm, g);
        if (!defer) {
          q = g.q;
          x = (T)g.x;
          y = (T)g.y;
          c2 = (T)g.c2b;
          s2 = (T)g.s2b;
        }
      } else {
        Geo g;
        const double z = rt.z[loc.ring], s = rt.sint[loc.ring];
        geo64(rt, nside, p, rt.theta[loc.ring], z, s, ring_phi(rt, loc.ring, loc.idx), (double)ath, (double)aph, rot,
              mode, g);
        q = g.q;
        x = (T)(Lnorm * g.dth);
        y = (T)(Lnorm * g.dph);
        c2 = (T)g.c2b;
        s2 = (T)g.s2b;
      }
    }
    if (defer)
      s_list[atomicAdd(&s_cnt, 1)] = (int)p;
    else
      taylor_store<T, ORDER, POL>(tile, p, q, x, y, c2, s2, d3, Tout, Qout, Uout);
  }
  if (FAST) {
    __syncthreads();
    const int n = s_cnt;
    if (n == 0) return;  // uniform
    if (threadIdx.x == 0) s_base = atomicAdd(qcount, n);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) queue[s_base + i] = s_list[i];
  }
}

// The deferred pixels of the float kernel, with the double geometry (grid-stride
// over the queue, whose length the device holds).
template <int ORDER, bool POL>
__global__ void __launch_bounds__(256) gather_fallback_kernel(RingTable rt, int nside, long long npix, double Lnorm,
                                                              const float *__restrict__ a_th,
                                                              const float *__restrict__ a_ph,
                                                              const float *__restrict__ d3, float *__restrict__ Tout,
                                                              float *__restrict__ Qout, float *__restrict__ Uout,
                                                              int rotate, const int *__restrict__ queue,
                                                              const int *__restrict__ qcount, long long tile,
                                                              int mode) {
  const int n = *qcount;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long p = queue[i];
    const PixLoc loc = pix2loc(p, nside, npix);
    Geo g;
    const double z = rt.z[loc.ring], s = rt.sint[loc.ring];
    geo64(rt, nside, p, rt.theta[loc.ring], z, s, ring_phi(rt, loc.ring, loc.idx), (double)a_th[p], (double)a_ph[p],
          POL && rotate, mode, g);
    taylor_store<float, ORDER, POL>(tile, p, g.q, (float)(Lnorm * g.dth), (float)(Lnorm * g.dph), (float)g.c2b,
                                    (float)g.s2b, d3, Tout, Qout, Uout);
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
  const int mode = ((p->flags & TL_NAIVE) ? kGeoNaive : 0) | ((p->flags & TL_EXPAND_AT_PIXEL) ? kGeoAtPixel : 0);
  const double L = (double)(p->lmax + 1);
  constexpr bool F32 = sizeof(T) == 4;
  constexpr int NM = (ORDER + 1) * (ORDER + 2) / 2;
  const long long tile = (long long)(pol ? 3 : 1) * NM * kD3Tile;  // d3's tile stride
  if (F32) {
    cudaError_t e = cudaMemsetAsync(p->gq_count, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  if (pol)
    gather_kernel<T, ORDER, true><<<(unsigned)blocks, threads, 0, s>>>(p->ring, p->nside, p->npix, L, ath, aph,
                                                                       (const T *)d3, (T *)Tq, (T *)Q, (T *)U, rot,
                                                                       p->gq, p->gq_count, tile, mode);
  else
    gather_kernel<T, ORDER, false><<<(unsigned)blocks, threads, 0, s>>>(p->ring, p->nside, p->npix, L, ath, aph,
                                                                        (const T *)d3, (T *)Tq, nullptr, nullptr,
                                                                        rot, p->gq, p->gq_count, tile, mode);
  if (F32) {
    // a fixed grid: the queue's length is known only on the device
    const int fb = 4 * p->num_sms;
    if (pol)
      gather_fallback_kernel<ORDER, true><<<fb, threads, 0, s>>>(
          p->ring, p->nside, p->npix, L, (const float *)ath, (const float *)aph, (const float *)d3, (float *)Tq,
          (float *)Q, (float *)U, rot, p->gq, p->gq_count, tile, mode);
    else
      gather_fallback_kernel<ORDER, false><<<fb, threads, 0, s>>>(
          p->ring, p->nside, p->npix, L, (const float *)ath, (const float *)aph, (const float *)d3, (float *)Tq,
          nullptr, nullptr, rot, p->gq, p->gq_count, tile, mode);
  }
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
