// Adjoint of the gather + Taylor + rotate step (Naess & Louis 2013, Eq. 4 and
// the rotation R of Eq. 2), one thread per output pixel p, with the expansion
// pixel q(p) held fixed (the lensed map is piecewise smooth in the deflection;
// q is constant between its jumps). For upstream gradients g_s(p), s in {T, Q, U}:
//   rotation:  (Q', U') = R(beta)(Q~, U~)   ->  (gQ~, gU~) = R(beta)^T (gQ, gU),
//              dL/dbeta = 2 (gQ U' - gU Q');
//   Eq. 4:     s~(p) = sum_{j,k} x^j y^k D~_jk(q),  x = L dth, y = L dph
//              ->  Dbar_jk[q] += x^j y^k g_s~  (atomic: several p share a q),
//              dL/d(dth) = L sum_s g_s~ ds~/dx,  dL/d(dph) = L sum_s g_s~ ds~/dy;
//   geometry:  (dth, dph, beta) as functions of (a_theta, a_phi) at fixed q
//              ->  galpha = J^T (dL/d(dth), dL/d(dph), dL/dbeta).
// The Jacobian J comes from forward-mode dual numbers through the double-precision
// geometry, written in a frame turned to the pixel's longitude and in terms of
// smooth functions of |alpha|^2, so that it is exact and regular at alpha = 0.
#include <math.h>

#include "geometry.cuh"

namespace tl {

// value and partial derivatives with respect to (a_theta, a_phi)
struct Dual {
  double v, a, b;
};
__device__ __forceinline__ Dual dconst(double v) { return Dual{v, 0.0, 0.0}; }
__device__ __forceinline__ Dual operator+(Dual x, Dual y) { return Dual{x.v + y.v, x.a + y.a, x.b + y.b}; }
__device__ __forceinline__ Dual operator-(Dual x, Dual y) { return Dual{x.v - y.v, x.a - y.a, x.b - y.b}; }
__device__ __forceinline__ Dual operator-(Dual x) { return Dual{-x.v, -x.a, -x.b}; }
__device__ __forceinline__ Dual operator*(Dual x, Dual y) {
  return Dual{x.v * y.v, x.a * y.v + x.v * y.a, x.b * y.v + x.v * y.b};
}
__device__ __forceinline__ Dual operator*(double c, Dual x) { return Dual{c * x.v, c * x.a, c * x.b}; }
__device__ __forceinline__ Dual operator/(Dual x, Dual y) {
  const double q = x.v / y.v;
  return Dual{q, (x.a - q * y.a) / y.v, (x.b - q * y.b) / y.v};
}
__device__ __forceinline__ Dual dhypot(Dual x, Dual y) {
  const double h = hypot(x.v, y.v);
  return Dual{h, (x.v * x.a + y.v * y.a) / h, (x.v * x.b + y.v * y.b) / h};
}
__device__ __forceinline__ Dual datan2(Dual y, Dual x) {
  const double d = x.v * x.v + y.v * y.v;
  return Dual{atan2(y.v, x.v), (x.v * y.a - y.v * x.a) / d, (x.v * y.b - y.v * x.b) / d};
}
// f(u) with f' given, u a dual
__device__ __forceinline__ Dual dfun(Dual u, double f, double fp) { return Dual{f, fp * u.a, fp * u.b}; }

// With u = d^2: S(u) = sin(d)/d, H(u) = (1 - cos d)/d^2, C(u) = cos d = 1 - u H,
// and their u-derivatives S' = (cos d - S)/(2u), H' = (S/2 - H)/u, C' = -S/2.
// Below u = 0.01 the Taylor series in u (truncation below 1e-20) replace the
// quotients, which lose digits there.
__device__ __forceinline__ void sinc_family(double u, double &S, double &Sp, double &H, double &Hp, double &C,
                                            double &Cp) {
  if (u < 0.01) {
    S = 1.0 + u * (-1.0 / 6 + u * (1.0 / 120 + u * (-1.0 / 5040 + u * (1.0 / 362880 + u * (-1.0 / 39916800)))));
    Sp = -1.0 / 6 + u * (1.0 / 60 + u * (-1.0 / 1680 + u * (1.0 / 90720 + u * (-1.0 / 7983360))));
    H = 0.5 + u * (-1.0 / 24 + u * (1.0 / 720 + u * (-1.0 / 40320 + u * (1.0 / 3628800 + u * (-1.0 / 479001600)))));
    Hp = -1.0 / 24 + u * (1.0 / 360 + u * (-1.0 / 13440 + u * (1.0 / 907200 + u * (-1.0 / 95800320))));
    C = 1.0 - u * H;
  } else {
    const double d = sqrt(u);
    double sd, cd;
    sincos(d, &sd, &cd);
    const double sh = sin(0.5 * d);
    S = sd / d;
    C = cd;
    H = 2.0 * sh * sh / u;
    Sp = (cd - S) / (2.0 * u);
    Hp = (0.5 * S - H) / u;
  }
  Cp = -0.5 * S;
}

struct GeoAdj {
  long long q;
  double dth, dph, c2b, s2b;
  double jth[2], jph[2], jb[2];  // d(dth), d(dph), d(beta) / d(a_theta, a_phi)
};

// Displaced point x' = C n + S (a_th e_th + a_ph e_ph) in the frame turned to the
// pixel's longitude (n = (s, 0, z), e_th = (z, 0, -s), e_ph = (0, 1, 0)); the
// transported e_theta(x) is t = (1 - a_th^2 H) e_th - a_th a_ph H e_ph - S a_th n.
__device__ __forceinline__ void geo_adj(const RingTable &rt, int nside, double z, double s, double phi, double ath_v,
                                        double aph_v, bool rot, GeoAdj &g) {
  const Dual ath{ath_v, 1.0, 0.0}, aph{aph_v, 0.0, 1.0};
  const Dual u = ath * ath + aph * aph;
  double S0, Sp, H0, Hp, C0, Cp;
  sinc_family(u.v, S0, Sp, H0, Hp, C0, Cp);
  const Dual S = dfun(u, S0, Sp), H = dfun(u, H0, Hp), C = dfun(u, C0, Cp);
  const Dual nx = s * C + z * (S * ath);
  const Dual ny = S * aph;
  const Dual nz = z * C - s * (S * ath);
  const Dual rho = dhypot(nx, ny);
  const Dual th2 = datan2(rho, nz);
  const Dual dphi = datan2(ny, nx);  // phi' - phi
  double phi2 = phi + dphi.v;
  if (phi2 >= 2.0 * kPiD) phi2 -= 2.0 * kPiD;
  if (phi2 < 0.0) phi2 += 2.0 * kPiD;
  const PixLoc lq = ang2loc(nz.v, rho.v * rho.v / (1.0 + fabs(nz.v)), phi2, nside);
  g.q = rt.first[lq.ring] + lq.idx;
  g.dth = th2.v - rt.theta[lq.ring];
  double dph = phi2 - ring_phi(rt, lq.ring, lq.idx);
  if (dph >= kPiD) dph -= 2.0 * kPiD;
  if (dph < -kPiD) dph += 2.0 * kPiD;
  g.dph = dph;
  g.jth[0] = th2.a;
  g.jth[1] = th2.b;
  g.jph[0] = dphi.a;
  g.jph[1] = dphi.b;
  g.c2b = 1.0;
  g.s2b = 0.0;
  g.jb[0] = g.jb[1] = 0.0;
  if (rot) {
    const Dual ct = dconst(1.0) - (ath * ath) * H;
    const Dual tx = z * ct - s * (S * ath);
    const Dual ty = -((ath * aph) * H);
    const Dual tz = -(s * ct) - z * (S * ath);
    const Dual cb = nz * (tx * nx + ty * ny) / rho - tz * rho;  // t . e_theta'
    const Dual sb = (ty * nx - tx * ny) / rho;                  // t . e_phi'
    const Dual beta = datan2(sb, cb);
    const double nrm = cb.v * cb.v + sb.v * sb.v;
    g.c2b = (cb.v * cb.v - sb.v * sb.v) / nrm;
    g.s2b = 2.0 * cb.v * sb.v / nrm;
    g.jb[0] = beta.a;
    g.jb[1] = beta.b;
  }
}

// Taylor sum of one field at q, its x- and y-derivatives, and the scatter of
// x^j y^k g into Dbar (all maps of the field, map index (j+k)(j+k+1)/2 + j). D: the
// field's first map in the pixel-tiled layout of the forward maps (tile: elements
// between tiles); Dbar: plain maps [map][npix].
template <typename T, int ORDER>
__device__ __forceinline__ void taylor_adj(const T *__restrict__ D, long long tile, T *__restrict__ Dbar,
                                           long long npix, long long q, const double (&xp)[ORDER + 1],
                                           const double (&yp)[ORDER + 1], double gs, double &val, double &dx,
                                           double &dy) {
  const long long qoff = d3_pix(q, tile);
  val = dx = dy = 0.0;
#pragma unroll
  for (int n = 0; n <= ORDER; ++n)
#pragma unroll
    for (int j = 0; j <= n; ++j) {
      const int k = n - j;
      const int mi = n * (n + 1) / 2 + j;
      const double d = (double)__ldg(D + qoff + (long long)mi * kD3Tile);
      val += xp[j] * yp[k] * d;
      if (j > 0) dx += (double)j * xp[j - 1] * yp[k] * d;
      if (k > 0) dy += (double)k * xp[j] * yp[k - 1] * d;
      if (gs != 0.0) atomicAdd(Dbar + (long long)mi * npix + q, (T)(xp[j] * yp[k] * gs));
    }
}

template <typename T, int ORDER, bool POL>
__global__ void __launch_bounds__(256) gather_adj_kernel(RingTable rt, int nside, long long npix, double Lnorm,
                                                         const T *__restrict__ a_th, const T *__restrict__ a_ph,
                                                         const T *__restrict__ d3, const T *__restrict__ gT,
                                                         const T *__restrict__ gQ, const T *__restrict__ gU,
                                                         T *__restrict__ dbar, T *__restrict__ ga_th,
                                                         T *__restrict__ ga_ph, int rotate) {
  constexpr int NM = (ORDER + 1) * (ORDER + 2) / 2;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npix) return;
  const PixLoc loc = pix2loc(p, nside, npix);
  const double z = rt.z[loc.ring], s = rt.sint[loc.ring];
  const double phi = ring_phi(rt, loc.ring, loc.idx);
  const bool rot = POL && rotate;
  GeoAdj g;
  geo_adj(rt, nside, z, s, phi, (double)a_th[p], (double)a_ph[p], rot, g);
  double xp[ORDER + 1], yp[ORDER + 1];
  const double x = Lnorm * g.dth, y = Lnorm * g.dph;
  xp[0] = yp[0] = 1.0;
#pragma unroll
  for (int i = 1; i <= ORDER; ++i) {
    xp[i] = xp[i - 1] * x;
    yp[i] = yp[i - 1] * y;
  }
  double v, dx, dy, dLdx = 0.0, dLdy = 0.0, dLdb = 0.0;
  const double gt = (double)gT[p];
  const long long tile = (long long)(POL ? 3 : 1) * NM * kD3Tile;  // forward maps' tile stride
  taylor_adj<T, ORDER>(d3, tile, dbar, npix, g.q, xp, yp, gt, v, dx, dy);
  dLdx += gt * dx;
  dLdy += gt * dy;
  if (POL) {
    const double gq = (double)gQ[p], gu = (double)gU[p];
    const double c2 = g.c2b, s2 = g.s2b;
    const double gqt = c2 * gq - s2 * gu, gut = s2 * gq + c2 * gu;
    double qv, qx, qy, uv, ux, uy;
    taylor_adj<T, ORDER>(d3 + NM * kD3Tile, tile, dbar + (long long)NM * npix, npix, g.q, xp, yp, gqt, qv, qx, qy);
    taylor_adj<T, ORDER>(d3 + 2 * NM * kD3Tile, tile, dbar + 2LL * NM * npix, npix, g.q, xp, yp, gut, uv, ux, uy);
    dLdx += gqt * qx + gut * ux;
    dLdy += gqt * qy + gut * uy;
    if (rot) {
      const double Qp = c2 * qv + s2 * uv, Up = -s2 * qv + c2 * uv;
      dLdb = 2.0 * (gq * Up - gu * Qp);
    }
  }
  const double dLdth = Lnorm * dLdx, dLdph = Lnorm * dLdy;
  ga_th[p] = (T)(dLdth * g.jth[0] + dLdph * g.jph[0] + dLdb * g.jb[0]);
  ga_ph[p] = (T)(dLdth * g.jth[1] + dLdph * g.jph[1] + dLdb * g.jb[1]);
}

template <typename T, int ORDER>
static cudaError_t gather_adj_t(const tl_plan *p, const void *alpha, const void *d3, const void *gT, const void *gQ,
                                const void *gU, void *dbar, void *ga, cudaStream_t s) {
  const int threads = 256;
  const long long blocks = (p->npix + threads - 1) / threads;
  const T *ath = (const T *)alpha;
  const T *aph = ath + p->npix;
  T *gath = (T *)ga;
  T *gaph = gath + p->npix;
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  const int rot = (p->flags & TL_ROTATE) ? 1 : 0;
  const double L = (double)(p->lmax + 1);
  if (pol)
    gather_adj_kernel<T, ORDER, true><<<(unsigned)blocks, threads, 0, s>>>(
        p->ring, p->nside, p->npix, L, ath, aph, (const T *)d3, (const T *)gT, (const T *)gQ, (const T *)gU,
        (T *)dbar, gath, gaph, rot);
  else
    gather_adj_kernel<T, ORDER, false><<<(unsigned)blocks, threads, 0, s>>>(
        p->ring, p->nside, p->npix, L, ath, aph, (const T *)d3, (const T *)gT, nullptr, nullptr, (T *)dbar, gath,
        gaph, rot);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t gather_adj_dispatch(const tl_plan *p, const void *a, const void *d3, const void *gT,
                                       const void *gQ, const void *gU, void *dbar, void *ga, cudaStream_t s) {
  switch (p->order) {
    case 0: return gather_adj_t<T, 0>(p, a, d3, gT, gQ, gU, dbar, ga, s);
    case 1: return gather_adj_t<T, 1>(p, a, d3, gT, gQ, gU, dbar, ga, s);
    case 2: return gather_adj_t<T, 2>(p, a, d3, gT, gQ, gU, dbar, ga, s);
    case 3: return gather_adj_t<T, 3>(p, a, d3, gT, gQ, gU, dbar, ga, s);
    case 4: return gather_adj_t<T, 4>(p, a, d3, gT, gQ, gU, dbar, ga, s);
    case 5: return gather_adj_t<T, 5>(p, a, d3, gT, gQ, gU, dbar, ga, s);
    case 6: return gather_adj_t<T, 6>(p, a, d3, gT, gQ, gU, dbar, ga, s);
  }
  return cudaErrorInvalidValue;
}

// dbar must be zeroed by the caller; ga receives [2][npix] (a_theta, a_phi gradients).
cudaError_t launch_gather_adjoint(const tl_plan *p, const void *alpha, const void *d3, const void *gT, const void *gQ,
                                  const void *gU, void *dbar, void *ga, cudaStream_t s) {
  return p->precision == TL_FP64 ? gather_adj_dispatch<double>(p, alpha, d3, gT, gQ, gU, dbar, ga, s)
                                 : gather_adj_dispatch<float>(p, alpha, d3, gT, gQ, gU, dbar, ga, s);
}

}  // namespace tl
