// Legendre stage kernels and coefficient preparation. See legendre.cuh for the
// mathematics (Naess & Louis 2013, Sec. II.B, Eq. 4 derivative maps).
#include <math.h>

#include "legendre.cuh"

namespace tl {

// ---------------------------------------------------------------------------
// coefficient preparation

__device__ __forceinline__ double rec_alpha(int L, int m, int s) {
  double L2 = (double)L * L;
  return sqrt((4.0 * L2 - 1.0) * L2 / ((L2 - (double)m * m) * (L2 - (double)s * s)));
}

template <typename T>
__global__ void prep_spin0_kernel(int lmax, const double *__restrict__ alm, Rec0<T> *__restrict__ rec) {
  int m = blockIdx.y;
  int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  long long idx = (long long)m * (2 * lmax + 1 - m) / 2 + l;
  Rec0<T> r;
  r.re = (T)alm[2 * idx];
  r.im = (m == 0) ? (T)0 : (T)alm[2 * idx + 1];
  if (l < lmax) {
    double an = rec_alpha(l + 1, m, 0);
    r.alpha = (T)an;
    r.beta = (l > m) ? (T)(an / rec_alpha(l, m, 0)) : (T)0;
  } else {
    r.alpha = (T)0;
    r.beta = (T)0;
  }
  rec[idx] = r;
}

template <typename T>
__global__ void prep_spin2_kernel(int lmax, const double *__restrict__ almE, const double *__restrict__ almB,
                                  Rec2<T> *__restrict__ rec) {
  int m = blockIdx.y;
  int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  long long idx = (long long)m * (2 * lmax + 1 - m) / 2 + l;
  const int s = 2;
  int l0 = m > s ? m : s;
  Rec2<T> r;
  if (l < l0) {
    r.c1r = r.c1i = r.c2r = r.c2i = r.alpha = r.beta = r.cterm = r.pad = (T)0;
    rec[idx] = r;
    return;
  }
  double er = almE ? almE[2 * idx] : 0.0;
  double ei = (almE && m > 0) ? almE[2 * idx + 1] : 0.0;
  double br = almB ? almB[2 * idx] : 0.0;
  double bi = (almB && m > 0) ? almB[2 * idx + 1] : 0.0;
  double sg = ((l + m) & 1) ? -1.0 : 1.0;
  r.c1r = (T)(er - bi);
  r.c1i = (T)(ei + br);
  r.c2r = (T)(sg * (er + bi));
  r.c2i = (T)(sg * (ei - br));
  if (l < lmax) {
    double an = rec_alpha(l + 1, m, s);
    r.alpha = (T)an;
    r.beta = (l > l0) ? (T)(an / rec_alpha(l, m, s)) : (T)0;
  } else {
    r.alpha = (T)0;
    r.beta = (T)0;
  }
  r.cterm = (T)((double)m * s / ((double)l * (l + 1.0)));
  r.pad = (T)0;
  rec[idx] = r;
}

// ---------------------------------------------------------------------------
// seeds

// Binomial coefficient, small arguments, compile-time friendly.
__host__ __device__ constexpr int binom(int n, int k) {
  return (k < 0 || k > n) ? 0 : (k == 0 || k == n) ? 1 : binom(n - 1, k - 1) + binom(n - 1, k);
}

// Seed mantissas (normalised derivatives) of s_lambda_{l0,m} at ring r.
// E = log2 |lambda|, exponents (a, b) of sin(th/2), cos(th/2), sign.
template <typename T, int NDER>
__device__ __forceinline__ void seed_values(const RingTable &rt, int r, double E, double a, double b,
                                            double sign, double invL, T (&cur)[NDER + 1], int &sc) {
  typedef RealTraits<T> RT;
  // scale: E - SB*sc in (H - SB, H]
  int s0 = (int)ceil((E - RT::H) / (double)RT::SB);
  if (s0 > 0) s0 = 0;
  sc = s0;
  double mant = sign * exp2(E - (double)RT::SB * s0);
  // d^j/dth^j f = f * B_j, B_{j+1} = sum_i C(j,i) g_{i+1} B_{j-i}
  double g[NDER + 1];
  const double *dls = rt.dls + (size_t)r * (TL_MAX_NDER + 1);
  const double *dlc = rt.dlc + (size_t)r * (TL_MAX_NDER + 1);
#pragma unroll
  for (int k = 1; k <= NDER; ++k) g[k] = a * dls[k - 1] + b * dlc[k - 1];
  double B[NDER + 1];
  B[0] = 1.0;
#pragma unroll
  for (int j = 0; j < NDER; ++j) {
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i <= j; ++i) acc += (double)binom(j, i) * g[i + 1] * B[j - i];
    B[j + 1] = acc;
  }
  double p = 1.0;
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    cur[j] = (T)(mant * B[j] * p);
    p *= invL;
  }
}

// Leibniz step: nxt^(j) = alpha (X cur^(j) + sum_{i>=1} e[j][i] cur^(j-i)) - beta prev^(j)
template <typename T, int NDER>
__device__ __forceinline__ void rec_step(T (&cur)[NDER + 1], T (&prev)[NDER + 1], const T (&dcos)[NDER + 1],
                                         T X, T alpha, T beta) {
  T nxt[NDER + 1];
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    T acc = X * cur[j];
#pragma unroll
    for (int i = 1; i <= j; ++i) acc = fma((T)binom(j, i) * dcos[i], cur[j - i], acc);
    nxt[j] = fma(alpha, acc, -beta * prev[j]);
  }
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    prev[j] = cur[j];
    cur[j] = nxt[j];
  }
}

template <typename T, int NDER>
__device__ __forceinline__ void maybe_rescale(T (&cur)[NDER + 1], T (&prev)[NDER + 1], int &sc) {
  typedef RealTraits<T> RT;
  const T thr = (T)exp2(RT::H);
  if (sc < 0 && fabs(cur[0]) > thr) {
    const T f = (T)exp2(-(double)RT::SB);
#pragma unroll
    for (int j = 0; j <= NDER; ++j) {
      cur[j] *= f;
      prev[j] *= f;
    }
    ++sc;
  }
}

// normalised derivatives of cos(theta): dcos[i] = cos(th + i pi/2) / L^i
template <typename T, int NDER>
__device__ __forceinline__ void cos_derivs(double x, double st, double invL, T (&dcos)[NDER + 1]) {
  double p = 1.0;
#pragma unroll
  for (int i = 0; i <= NDER; ++i) {
    double v = (i % 4 == 0) ? x : (i % 4 == 1) ? -st : (i % 4 == 2) ? -x : st;
    dcos[i] = (T)(v * p);
    p *= invL;
  }
}

// ---------------------------------------------------------------------------
// spin 0: one thread per north ring (incl. the equator) and one m per block
// row; the south ring follows from lam^(j)(pi - th) = (-1)^(l+m+j) lam^(j)(th).

template <typename T, int NDER>
__global__ void __launch_bounds__(128) legendre_spin0_kernel(RingTable rt, const double *__restrict__ lnorm0,
                                                             int nside, int lmax, int mmax, int nrings,
                                                             const Rec0<T> *__restrict__ rec,
                                                             typename RealTraits<T>::T2 *__restrict__ d7) {
  typedef typename RealTraits<T>::T2 T2;
  const int m = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;  // north ring index 0 .. 2N-1
  if (r >= 2 * nside) return;
  const double invL = 1.0 / (double)(lmax + 1);
  const double x = rt.z[r], st = rt.sint[r];
  T dcos[NDER + 1];
  cos_derivs<T, NDER>(x, st, invL, dcos);

  T cur[NDER + 1], prev[NDER + 1];
  int sc;
  {
    double E = lnorm0[m] + (double)m * (rt.log2_sh[r] + rt.log2_ch[r]);
    seed_values<T, NDER>(rt, r, E, (double)m, (double)m, (m & 1) ? -1.0 : 1.0, invL, cur, sc);
  }
#pragma unroll
  for (int j = 0; j <= NDER; ++j) prev[j] = (T)0;

  // accumulators: even / odd l-m, real / imaginary
  T ae_r[NDER + 1], ae_i[NDER + 1], ao_r[NDER + 1], ao_i[NDER + 1];
#pragma unroll
  for (int j = 0; j <= NDER; ++j) ae_r[j] = ae_i[j] = ao_r[j] = ao_i[j] = (T)0;

  const Rec0<T> *rm = rec + (long long)m * (2 * lmax + 1 - m) / 2;
  const T X = (T)x;
  for (int l = m; l <= lmax; l += 2) {
    // even l - m
    {
      Rec0<T> c = rm[l];
      if (sc == 0) {
#pragma unroll
        for (int j = 0; j <= NDER; ++j) {
          ae_r[j] = fma(c.re, cur[j], ae_r[j]);
          ae_i[j] = fma(c.im, cur[j], ae_i[j]);
        }
      }
      if (l == lmax) break;
      rec_step<T, NDER>(cur, prev, dcos, X, c.alpha, c.beta);
      maybe_rescale<T, NDER>(cur, prev, sc);
    }
    // odd l - m
    {
      Rec0<T> c = rm[l + 1];
      if (sc == 0) {
#pragma unroll
        for (int j = 0; j <= NDER; ++j) {
          ao_r[j] = fma(c.re, cur[j], ao_r[j]);
          ao_i[j] = fma(c.im, cur[j], ao_i[j]);
        }
      }
      if (l + 1 == lmax) break;
      rec_step<T, NDER>(cur, prev, dcos, X, c.alpha, c.beta);
      maybe_rescale<T, NDER>(cur, prev, sc);
    }
  }
  if (m > mmax) return;
  const int rs = nrings - 1 - r;
  const size_t ld = (size_t)(mmax + 1);
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    T2 vn, vs;
    vn.x = ae_r[j] + ao_r[j];
    vn.y = ae_i[j] + ao_i[j];
    T sgn = (j & 1) ? (T)-1 : (T)1;
    vs.x = sgn * (ae_r[j] - ao_r[j]);
    vs.y = sgn * (ae_i[j] - ao_i[j]);
    d7[((size_t)j * nrings + r) * ld + m] = vn;
    if (rs != r) d7[((size_t)j * nrings + rs) * ld + m] = vs;
  }
}

// ---------------------------------------------------------------------------
// spin 2: block = 2 x RP threads; the first RP threads take north rings
// r0 .. r0+RP-1, the other RP their mirror rings pi - theta. Each thread runs
// the spin-2 recurrence on its own ring and accumulates
//   S1^(j) = sum_l (E + iB) 2lam^(j),  S2^(j) = sum_l (-1)^(l+m) (E - iB) 2lam^(j);
// with -2lam^(j)(th) = (-1)^(l+m+j) 2lam^(j)(pi - th), the pair combines into
//   F^Q(th) = -(S1(th) + (-1)^j S2(pi-th))/2,  F^U(th) = i (S1(th) - (-1)^j S2(pi-th))/2.

template <typename T, int NDER, int RP>
__global__ void __launch_bounds__(2 * RP) legendre_spin2_kernel(RingTable rt, const double *__restrict__ lnorm0,
                                                                int nside, int lmax, int mmax, int nrings,
                                                                const Rec2<T> *__restrict__ rec,
                                                                typename RealTraits<T>::T2 *__restrict__ d7q,
                                                                typename RealTraits<T>::T2 *__restrict__ d7u) {
  typedef typename RealTraits<T>::T2 T2;
  __shared__ T2 xch[2 * RP][NDER + 1];
  const int m = blockIdx.y;
  const int t = threadIdx.x;
  const int rn = blockIdx.x * RP + (t % RP);  // north ring of the pair
  const bool active = rn < 2 * nside;
  const bool mirror = t >= RP;
  const int r = active ? (mirror ? nrings - 1 - rn : rn) : 0;
  const double invL = 1.0 / (double)(lmax + 1);

  T s1r[NDER + 1], s1i[NDER + 1], s2r[NDER + 1], s2i[NDER + 1];
#pragma unroll
  for (int j = 0; j <= NDER; ++j) s1r[j] = s1i[j] = s2r[j] = s2i[j] = (T)0;

  if (active) {
    const double x = rt.z[r], st = rt.sint[r];
    T dcos[NDER + 1];
    cos_derivs<T, NDER>(x, st, invL, dcos);
    T cur[NDER + 1], prev[NDER + 1];
    int sc;
    int l0;
    {
      const double lsh = rt.log2_sh[r], lch = rt.log2_ch[r];
      double E, a, b;
      if (m >= 2) {
        l0 = m;
        double md = (double)m;
        E = lnorm0[m] + 0.5 * log2(md * (md - 1.0) / ((md + 1.0) * (md + 2.0))) + (md + 2.0) * lsh +
            (md - 2.0) * lch;
        a = md + 2.0;
        b = md - 2.0;
      } else {
        l0 = 2;
        // sqrt(5/(4 pi)) sqrt(C(4, 2+m))
        double c4 = (m == 0) ? 6.0 : 4.0;
        E = log2(sqrt(5.0 / (4.0 * 3.14159265358979323846)) * sqrt(c4)) + (2.0 + m) * lsh + (2.0 - m) * lch;
        a = 2.0 + m;
        b = 2.0 - m;
      }
      seed_values<T, NDER>(rt, r, E, a, b, (m & 1) ? -1.0 : 1.0, invL, cur, sc);
    }
#pragma unroll
    for (int j = 0; j <= NDER; ++j) prev[j] = (T)0;
    const Rec2<T> *rm = rec + (long long)m * (2 * lmax + 1 - m) / 2;
    const T X = (T)x;
    for (int l = l0; l <= lmax; ++l) {
      const Rec2<T> c = rm[l];
      if (sc == 0) {
#pragma unroll
        for (int j = 0; j <= NDER; ++j) {
          s1r[j] = fma(c.c1r, cur[j], s1r[j]);
          s1i[j] = fma(c.c1i, cur[j], s1i[j]);
          s2r[j] = fma(c.c2r, cur[j], s2r[j]);
          s2i[j] = fma(c.c2i, cur[j], s2i[j]);
        }
      }
      if (l == lmax) break;
      rec_step<T, NDER>(cur, prev, dcos, X + c.cterm, c.alpha, c.beta);
      maybe_rescale<T, NDER>(cur, prev, sc);
    }
  }
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    T2 v;
    v.x = s2r[j];
    v.y = s2i[j];
    xch[t][j] = v;
  }
  __syncthreads();
  if (!active || m > mmax) return;
  if (mirror && rn == nrings - 1 - rn) return;  // equator: the north thread writes it
  const int partner = mirror ? t - RP : t + RP;
  const size_t ld = (size_t)(mmax + 1);
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    T2 p = xch[partner][j];
    T sg = (j & 1) ? (T)-1 : (T)1;
    T ar = s1r[j] + sg * p.x, ai = s1i[j] + sg * p.y;  // S1 + (-1)^j S2'
    T br = s1r[j] - sg * p.x, bi = s1i[j] - sg * p.y;  // S1 - (-1)^j S2'
    T2 q, u;
    q.x = (T)-0.5 * ar;
    q.y = (T)-0.5 * ai;
    u.x = (T)-0.5 * bi;  // i (br + i bi)/2
    u.y = (T)0.5 * br;
    size_t o = ((size_t)j * nrings + r) * ld + m;
    d7q[o] = q;
    d7u[o] = u;
  }
}

// ---------------------------------------------------------------------------
// launchers

template <typename T>
static cudaError_t prep0(const tl_plan *p, const double *alm, void *rec, cudaStream_t s) {
  dim3 grid((p->lmax + 1 + 127) / 128, p->lmax + 1);
  prep_spin0_kernel<T><<<grid, 128, 0, s>>>(p->lmax, alm, (Rec0<T> *)rec);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t prep2(const tl_plan *p, const double *almE, const double *almB, void *rec, cudaStream_t s) {
  dim3 grid((p->lmax + 1 + 127) / 128, p->lmax + 1);
  prep_spin2_kernel<T><<<grid, 128, 0, s>>>(p->lmax, almE, almB, (Rec2<T> *)rec);
  return cudaGetLastError();
}

cudaError_t launch_prep_spin0(const tl_plan *p, const double *alm, void *rec, cudaStream_t s) {
  return p->precision == TL_FP64 ? prep0<double>(p, alm, rec, s) : prep0<float>(p, alm, rec, s);
}
cudaError_t launch_prep_spin2(const tl_plan *p, const double *almE, const double *almB, void *rec,
                              cudaStream_t s) {
  return p->precision == TL_FP64 ? prep2<double>(p, almE, almB, rec, s) : prep2<float>(p, almE, almB, rec, s);
}

template <typename T, int NDER>
static cudaError_t leg0(const tl_plan *p, const void *rec, void *d7, cudaStream_t s) {
  const int threads = 64;
  dim3 grid((2 * p->nside + threads - 1) / threads, p->mmax + 1);
  legendre_spin0_kernel<T, NDER><<<grid, threads, 0, s>>>(
      p->ring, p->lnorm0, p->nside, p->lmax, p->mmax, p->nrings, (const Rec0<T> *)rec,
      (typename RealTraits<T>::T2 *)d7);
  return cudaGetLastError();
}

template <typename T, int NDER>
static cudaError_t leg2(const tl_plan *p, const void *rec, void *dq, void *du, cudaStream_t s) {
  constexpr int RP = 32;
  dim3 grid((2 * p->nside + RP - 1) / RP, p->mmax + 1);
  legendre_spin2_kernel<T, NDER, RP><<<grid, 2 * RP, 0, s>>>(
      p->ring, p->lnorm0, p->nside, p->lmax, p->mmax, p->nrings, (const Rec2<T> *)rec,
      (typename RealTraits<T>::T2 *)dq, (typename RealTraits<T>::T2 *)du);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t leg0_dispatch(const tl_plan *p, int nder, const void *rec, void *d7, cudaStream_t s) {
  switch (nder) {
    case 0: return leg0<T, 0>(p, rec, d7, s);
    case 1: return leg0<T, 1>(p, rec, d7, s);
    case 2: return leg0<T, 2>(p, rec, d7, s);
    case 3: return leg0<T, 3>(p, rec, d7, s);
    case 4: return leg0<T, 4>(p, rec, d7, s);
    case 5: return leg0<T, 5>(p, rec, d7, s);
    case 6: return leg0<T, 6>(p, rec, d7, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t leg2_dispatch(const tl_plan *p, int nder, const void *rec, void *dq, void *du, cudaStream_t s) {
  switch (nder) {
    case 0: return leg2<T, 0>(p, rec, dq, du, s);
    case 1: return leg2<T, 1>(p, rec, dq, du, s);
    case 2: return leg2<T, 2>(p, rec, dq, du, s);
    case 3: return leg2<T, 3>(p, rec, dq, du, s);
    case 4: return leg2<T, 4>(p, rec, dq, du, s);
    case 5: return leg2<T, 5>(p, rec, dq, du, s);
    case 6: return leg2<T, 6>(p, rec, dq, du, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_legendre_spin0(const tl_plan *p, int nder, const void *rec, void *d7, cudaStream_t s) {
  return p->precision == TL_FP64 ? leg0_dispatch<double>(p, nder, rec, d7, s)
                                 : leg0_dispatch<float>(p, nder, rec, d7, s);
}

cudaError_t launch_legendre_spin2(const tl_plan *p, int nder, const void *rec, void *dq, void *du,
                                  cudaStream_t s) {
  return p->precision == TL_FP64 ? leg2_dispatch<double>(p, nder, rec, dq, du, s)
                                 : leg2_dispatch<float>(p, nder, rec, dq, du, s);
}

}  // namespace tl
