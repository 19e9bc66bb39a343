// Legendre stage kernels, their plan-time step tables and the per-call
// coefficient preparation. See legendre.cuh for the mathematics (Naess & Louis
// 2013, Sec. II.B: the derivative maps of Eq. 4).
//
// Normalised recurrence. With lam_l = k_l mu_l and k_{l+1} = beta_{l+1} k_{l-1}
// (k_{l0} = k_{l0+1} = 1) the three-term recurrence becomes
//     mu_{l+1} = A_{l+1} X mu_l - mu_{l-1},   A_{l+1} = alpha_{l+1} k_l / k_{l+1},
// so each step of each derivative order ends in one fused multiply-add; k_l is
// folded into the coefficients (sum_l a_l lam_l = sum_l (a_l k_l) mu_l). The
// table {k_l, A_{l+1}} depends only on (l, m, s) and is built once per plan.
#include <math.h>

#include "legendre.cuh"

namespace tl {

// ---------------------------------------------------------------------------
// step tables and coefficient preparation

__device__ __forceinline__ double rec_alpha(int L, int m, int s) {
  double L2 = (double)L * L;
  return sqrt((4.0 * L2 - 1.0) * L2 / ((L2 - (double)m * m) * (L2 - (double)s * s)));
}

// One thread per m: tab[idx(l, m)] = {k_l, A_{l+1} - 2} for l0 <= l <= lmax (A = 0,
// i.e. -2 stored, at lmax). k_{l0} = 1; k_{l0+1} = g is chosen so that the even
// and odd chains k_{l+1} = beta_{l+1} k_{l-1} end at the same value: a first pass
// runs them with g = 1 and takes g = (even chain) / (odd chain) at lmax, so the
// normalised step factor A tends to 2 without alternating about it.
template <typename T>
__global__ void steptab_kernel(int lmax, int s, typename RealTraits<T>::T2 *__restrict__ tab) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > lmax) return;
  const int as = s < 0 ? -s : s;
  const int l0 = m > as ? m : as;
  typename RealTraits<T>::T2 *tm = tab + (long long)m * (2 * lmax + 1 - m) / 2;
  for (int l = m; l < l0 && l <= lmax; ++l) {
    tm[l].x = (T)0;
    tm[l].y = (T)0;
  }
  if (l0 > lmax) return;
  double g = 1.0;
  if (lmax >= l0 + 2) {
    double k_prev = 1.0, k_cur = 1.0, a_cur = rec_alpha(l0 + 1, m, s);  // k_{l0}, k_{l0+1}, alpha_{l0+1}
    for (int l = l0 + 1; l < lmax; ++l) {
      const double a_next = rec_alpha(l + 1, m, s);
      const double k_next = (a_next / a_cur) * k_prev;
      k_prev = k_cur;
      k_cur = k_next;
      a_cur = a_next;
    }
    // k_cur = k_lmax, k_prev = k_{lmax-1}
    g = ((lmax - l0) % 2 == 0) ? k_cur / k_prev : k_prev / k_cur;
  }
  double k_prev = 1.0, k_cur = 1.0, a_cur = 0.0;  // k_{l-1}, k_l, alpha_l
  for (int l = l0; l <= lmax; ++l) {
    double Am2 = -2.0, k_next = 0.0;
    if (l < lmax) {
      const double a_next = rec_alpha(l + 1, m, s);
      k_next = (l == l0) ? g : (a_next / a_cur) * k_prev;  // beta_{l+1} k_{l-1}
      Am2 = a_next * k_cur / k_next - 2.0;
      a_cur = a_next;
    }
    tm[l].x = (T)k_cur;
    tm[l].y = (T)Am2;
    k_prev = k_cur;
    k_cur = k_next;
  }
}

template <typename T>
__global__ void prep_spin0_kernel(int lmax, const double *__restrict__ alm,
                                  const typename RealTraits<T>::T2 *__restrict__ tab, Rec0<T> *__restrict__ rec) {
  const int m = blockIdx.y;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  const long long idx = (long long)m * (2 * lmax + 1 - m) / 2 + l;
  const typename RealTraits<T>::T2 kA = tab[idx];
  Rec0<T> r;
  r.re = (T)(alm[2 * idx] * (double)kA.x);
  r.im = (m == 0) ? (T)0 : (T)(alm[2 * idx + 1] * (double)kA.x);
  r.A = (T)(2.0 + (double)kA.y);
  r.Q = kA.y;
  rec[idx] = r;
}

// coefficients of a second spin-0 field that shares the basis (the lensing potential)
template <typename T>
__global__ void prep_phi_kernel(int lmax, const double *__restrict__ alm,
                                const typename RealTraits<T>::T2 *__restrict__ tab,
                                typename RealTraits<T>::T2 *__restrict__ rec) {
  const int m = blockIdx.y;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  const long long idx = (long long)m * (2 * lmax + 1 - m) / 2 + l;
  const double k = (double)tab[idx].x;
  typename RealTraits<T>::T2 r;
  r.x = (T)(alm[2 * idx] * k);
  r.y = (m == 0) ? (T)0 : (T)(alm[2 * idx + 1] * k);
  rec[idx] = r;
}

template <typename T>
__global__ void prep_spin2_kernel(int lmax, const double *__restrict__ almE, const double *__restrict__ almB,
                                  const typename RealTraits<T>::T2 *__restrict__ tab, Rec2<T> *__restrict__ rec) {
  const int m = blockIdx.y;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  const long long idx = (long long)m * (2 * lmax + 1 - m) / 2 + l;
  const int s = 2;
  const int l0 = m > s ? m : s;
  Rec2<T> r;
  if (l < l0) {
    r.c1r = r.c1i = r.c2r = r.c2i = r.A = r.cterm = r.Qn = r.Qs = (T)0;
    rec[idx] = r;
    return;
  }
  const typename RealTraits<T>::T2 kA = tab[idx];
  const double k = (double)kA.x;
  const double er = almE ? almE[2 * idx] : 0.0;
  const double ei = (almE && m > 0) ? almE[2 * idx + 1] : 0.0;
  const double br = almB ? almB[2 * idx] : 0.0;
  const double bi = (almB && m > 0) ? almB[2 * idx + 1] : 0.0;
  const double sg = ((l + m) & 1) ? -k : k;
  r.c1r = (T)((er - bi) * k);
  r.c1i = (T)((ei + br) * k);
  r.c2r = (T)(sg * (er + bi));
  r.c2i = (T)(sg * (ei - br));
  const double Am2 = (double)kA.y, A = 2.0 + Am2, C = (double)m * s / ((double)l * (l + 1.0));
  r.A = (T)A;
  r.cterm = (T)C;
  r.Qn = (T)(Am2 + A * C);
  r.Qs = (T)(Am2 - A * C);
  rec[idx] = r;
}

// ---------------------------------------------------------------------------
// spin 0: one thread per north ring (incl. the equator) and one m per block
// row; the south ring follows from lam^(j)(pi - th) = (-1)^(l+m+j) lam^(j)(th),
// so even and odd l - m are accumulated apart. With PHI, the lensing potential's
// coefficients are contracted against the same basis for j <= 1 (deflection).

template <typename T, int NDER, bool PHI>
__global__ void __launch_bounds__(128) legendre_spin0_kernel(RingTable rt, const double *__restrict__ lnorm0,
                                                             int nside, int lmax, int mmax, int nrings,
                                                             const Rec0<T> *__restrict__ rec,
                                                             const typename RealTraits<T>::T2 *__restrict__ recp,
                                                             typename RealTraits<T>::T2 *__restrict__ d7,
                                                             typename RealTraits<T>::T2 *__restrict__ d7p) {
  typedef typename RealTraits<T>::T2 T2;
  constexpr int NP = PHI ? 2 : 0;  // phi derivative orders carried (0 and 1)
  const int m = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;  // north ring index 0 .. 2N-1
  if (r >= 2 * nside) return;
  const double invL = 1.0 / (double)(lmax + 1);
  const double x = rt.z[r], st = rt.sint[r];
  Leib<T, NDER> LC;
  leibniz_coefs<T, NDER>(x, st, invL, LC);

  T a[NDER + 1], b[NDER + 1];  // recurrence state: b = mu_l; a = d_l (float) or mu_{l-1} (double)
  int sc;
  seed_spin0<T, NDER>(rt, lnorm0, r, m, invL, b, sc);
  rec_init<T, NDER>(a, b);

  T er[NDER + 1], ei[NDER + 1], orr[NDER + 1], oi[NDER + 1];
#pragma unroll
  for (int j = 0; j <= NDER; ++j) er[j] = ei[j] = orr[j] = oi[j] = (T)0;
  T per[2], pei[2], por[2], poi[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) per[j] = pei[j] = por[j] = poi[j] = (T)0;

  const long long base = (long long)m * (2 * lmax + 1 - m) / 2;
  const Rec0<T> *rm = rec + base;
  const T2 *pm = PHI ? recp + base : nullptr;
  const T X = (T)x, w = (T)rt.omza[r];  // north rings: cos th >= 0
  Rec0<T> cn = rm[m];
  T2 pn;
  if (PHI) pn = pm[m];
  for (int l = m;; l += 2) {
    // ---- even l - m
    {
      const Rec0<T> c = cn;
      T2 pc;
      if (PHI) pc = pn;
      if (l + 1 <= lmax) {
        cn = rm[l + 1];
        if (PHI) pn = pm[l + 1];
      }
      if (sc == 0) {
#pragma unroll
        for (int j = 0; j <= NDER; ++j) {
          er[j] = fma(c.re, b[j], er[j]);
          ei[j] = fma(c.im, b[j], ei[j]);
        }
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          per[j] = fma(pc.x, b[j], per[j]);
          pei[j] = fma(pc.y, b[j], pei[j]);
        }
      }
      if (l == lmax) break;
      rec_step<T, NDER, 1>(a, b, LC, X, w, c.A, c.Q);
      rescale<T, NDER>(a, b, b[0], sc);
    }
    // ---- odd l - m
    {
      const Rec0<T> c = cn;
      T2 pc;
      if (PHI) pc = pn;
      if (l + 2 <= lmax) {
        cn = rm[l + 2];
        if (PHI) pn = pm[l + 2];
      }
      if (sc == 0) {
#pragma unroll
        for (int j = 0; j <= NDER; ++j) {
          orr[j] = fma(c.re, b[j], orr[j]);
          oi[j] = fma(c.im, b[j], oi[j]);
        }
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          por[j] = fma(pc.x, b[j], por[j]);
          poi[j] = fma(pc.y, b[j], poi[j]);
        }
      }
      if (l + 1 == lmax) break;
      rec_step<T, NDER, 1>(a, b, LC, X, w, c.A, c.Q);
      rescale<T, NDER>(a, b, b[0], sc);
    }
  }
  if (m > mmax) return;
  const int rs = nrings - 1 - r;
  const size_t ld = (size_t)(mmax + 1);
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    T2 vn, vs;
    vn.x = er[j] + orr[j];
    vn.y = ei[j] + oi[j];
    const T sgn = (j & 1) ? (T)-1 : (T)1;
    vs.x = sgn * (er[j] - orr[j]);
    vs.y = sgn * (ei[j] - oi[j]);
    d7[((size_t)j * nrings + r) * ld + m] = vn;
    if (rs != r) d7[((size_t)j * nrings + rs) * ld + m] = vs;
  }
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    T2 vn, vs;
    vn.x = per[j] + por[j];
    vn.y = pei[j] + poi[j];
    const T sgn = (j & 1) ? (T)-1 : (T)1;
    vs.x = sgn * (per[j] - por[j]);
    vs.y = sgn * (pei[j] - poi[j]);
    d7p[((size_t)j * nrings + r) * ld + m] = vn;
    if (rs != r) d7p[((size_t)j * nrings + rs) * ld + m] = vs;
  }
}

// ---------------------------------------------------------------------------
// spin 2: block = 2 x RP threads; the first RP threads take north rings
// r0 .. r0+RP-1, the other RP their mirror rings pi - theta. Each thread runs
// the spin-2 recurrence on its own ring and accumulates
//   S1^(j) = sum_l (E + iB) 2lam^(j),  S2^(j) = sum_l (-1)^(l+m) (E - iB) 2lam^(j);
// with -2lam^(j)(th) = (-1)^(l+m+j) 2lam^(j)(pi - th), the pair combines into
//   F^Q(th) = -(S1(th) + (-1)^j S2(pi-th))/2,  F^U(th) = i (S1(th) - (-1)^j S2(pi-th))/2.

template <typename T, int NDER>
__device__ __forceinline__ void acc2(const Rec2<T> &c, const T (&v)[NDER + 1], T (&s1r)[NDER + 1],
                                     T (&s1i)[NDER + 1], T (&s2r)[NDER + 1], T (&s2i)[NDER + 1]) {
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    s1r[j] = fma(c.c1r, v[j], s1r[j]);
    s1i[j] = fma(c.c1i, v[j], s1i[j]);
    s2r[j] = fma(c.c2r, v[j], s2r[j]);
    s2i[j] = fma(c.c2i, v[j], s2i[j]);
  }
}

// The recurrence of one ring from l0 to lmax, contracted as it goes (SG = sign cos th).
template <typename T, int NDER, int SG>
__device__ __forceinline__ void spin2_sweep(const Rec2<T> *__restrict__ rm, int l0, int lmax, const Leib<T, NDER> &LC,
                                            T X, T w, T (&a)[NDER + 1], T (&b)[NDER + 1], int &sc,
                                            T (&s1r)[NDER + 1], T (&s1i)[NDER + 1], T (&s2r)[NDER + 1],
                                            T (&s2i)[NDER + 1]) {
  Rec2<T> cn = rm[l0];
#pragma unroll 2
  for (int l = l0;; ++l) {
    const Rec2<T> c = cn;
    if (l + 1 <= lmax) cn = rm[l + 1];
    if (sc == 0) acc2<T, NDER>(c, b, s1r, s1i, s2r, s2i);
    if (l == lmax) break;
    rec_step<T, NDER, SG>(a, b, LC, X + c.cterm, w, c.A, SG > 0 ? c.Qn : c.Qs);
    rescale<T, NDER>(a, b, b[0], sc);
  }
}

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
    Leib<T, NDER> LC;
    leibniz_coefs<T, NDER>(x, st, invL, LC);
    T a[NDER + 1], b[NDER + 1];  // b = mu_l; a = d_l (float) or mu_{l-1} (double)
    int sc;
    const int l0 = seed_spin2<T, NDER>(rt, lnorm0, r, m, invL, b, sc);
    rec_init<T, NDER>(a, b);
    const Rec2<T> *rm = rec + (long long)m * (2 * lmax + 1 - m) / 2;
    const T X = (T)x, w = (T)rt.omza[r];
    if (l0 <= lmax) {
      // mirror threads (cos th < 0) are whole warps: RP is a multiple of 32
      if (mirror)
        spin2_sweep<T, NDER, -1>(rm, l0, lmax, LC, X, w, a, b, sc, s1r, s1i, s2r, s2i);
      else
        spin2_sweep<T, NDER, 1>(rm, l0, lmax, LC, X, w, a, b, sc, s1r, s1i, s2r, s2i);
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
    const T2 p = xch[partner][j];
    const T sg = (j & 1) ? (T)-1 : (T)1;
    const T ar = s1r[j] + sg * p.x, ai = s1i[j] + sg * p.y;  // S1 + (-1)^j S2'
    const T br = s1r[j] - sg * p.x, bi = s1i[j] - sg * p.y;  // S1 - (-1)^j S2'
    T2 q, u;
    q.x = (T)-0.5 * ar;
    q.y = (T)-0.5 * ai;
    u.x = (T)-0.5 * bi;  // i (br + i bi) / 2
    u.y = (T)0.5 * br;
    const size_t o = ((size_t)j * nrings + r) * ld + m;
    d7q[o] = q;
    d7u[o] = u;
  }
}

// ---------------------------------------------------------------------------
// launchers

template <typename T>
static cudaError_t steptab_t(int lmax, int s, void *tab, cudaStream_t st) {
  steptab_kernel<T><<<(lmax + 1 + 127) / 128, 128, 0, st>>>(lmax, s, (typename RealTraits<T>::T2 *)tab);
  return cudaGetLastError();
}
cudaError_t launch_steptab(const tl_plan *p, int s, void *tab, cudaStream_t st) {
  return p->precision == TL_FP64 ? steptab_t<double>(p->lmax, s, tab, st) : steptab_t<float>(p->lmax, s, tab, st);
}

template <typename T>
static cudaError_t prep0(const tl_plan *p, const double *alm, const double *alm_phi, cudaStream_t s) {
  typedef typename RealTraits<T>::T2 T2;
  dim3 grid((p->lmax + 1 + 127) / 128, p->lmax + 1);
  if (alm) prep_spin0_kernel<T><<<grid, 128, 0, s>>>(p->lmax, alm, (const T2 *)p->tab0, (Rec0<T> *)p->rec_T);
  if (alm_phi) prep_phi_kernel<T><<<grid, 128, 0, s>>>(p->lmax, alm_phi, (const T2 *)p->tab0, (T2 *)p->rec_P);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t prep2(const tl_plan *p, const double *almE, const double *almB, cudaStream_t s) {
  typedef typename RealTraits<T>::T2 T2;
  dim3 grid((p->lmax + 1 + 127) / 128, p->lmax + 1);
  prep_spin2_kernel<T><<<grid, 128, 0, s>>>(p->lmax, almE, almB, (const T2 *)p->tab2, (Rec2<T> *)p->rec_QU);
  return cudaGetLastError();
}

cudaError_t launch_prep_spin0(const tl_plan *p, const double *alm, const double *alm_phi, cudaStream_t s) {
  return p->precision == TL_FP64 ? prep0<double>(p, alm, alm_phi, s) : prep0<float>(p, alm, alm_phi, s);
}
cudaError_t launch_prep_spin2(const tl_plan *p, const double *almE, const double *almB, cudaStream_t s) {
  return p->precision == TL_FP64 ? prep2<double>(p, almE, almB, s) : prep2<float>(p, almE, almB, s);
}

template <typename T, int NDER, bool PHI>
static cudaError_t leg0(const tl_plan *p, void *d7, void *d7p, cudaStream_t s) {
  typedef typename RealTraits<T>::T2 T2;
  const int threads = 64;
  dim3 grid((2 * p->nside + threads - 1) / threads, p->mmax + 1);
  legendre_spin0_kernel<T, NDER, PHI><<<grid, threads, 0, s>>>(
      p->ring, p->lnorm0, p->nside, p->lmax, p->mmax, p->nrings, (const Rec0<T> *)p->rec_T,
      (const T2 *)p->rec_P, (T2 *)d7, (T2 *)d7p);
  return cudaGetLastError();
}

template <typename T, int NDER>
static cudaError_t leg2(const tl_plan *p, cudaStream_t s) {
  constexpr int RP = 32;
  dim3 grid((2 * p->nside + RP - 1) / RP, p->mmax + 1);
  legendre_spin2_kernel<T, NDER, RP><<<grid, 2 * RP, 0, s>>>(
      p->ring, p->lnorm0, p->nside, p->lmax, p->mmax, p->nrings, (const Rec2<T> *)p->rec_QU,
      (typename RealTraits<T>::T2 *)p->d7_Q, (typename RealTraits<T>::T2 *)p->d7_U);
  return cudaGetLastError();
}

template <typename T, bool PHI>
static cudaError_t leg0_dispatch(const tl_plan *p, int nder, void *d7, void *d7p, cudaStream_t s) {
  switch (nder) {
    case 0: return PHI ? cudaErrorInvalidValue : leg0<T, 0, false>(p, d7, d7p, s);
    case 1: return leg0<T, 1, PHI>(p, d7, d7p, s);
    case 2: return leg0<T, 2, PHI>(p, d7, d7p, s);
    case 3: return leg0<T, 3, PHI>(p, d7, d7p, s);
    case 4: return leg0<T, 4, PHI>(p, d7, d7p, s);
    case 5: return leg0<T, 5, PHI>(p, d7, d7p, s);
    case 6: return leg0<T, 6, PHI>(p, d7, d7p, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t leg2_dispatch(const tl_plan *p, int nder, cudaStream_t s) {
  switch (nder) {
    case 0: return leg2<T, 0>(p, s);
    case 1: return leg2<T, 1>(p, s);
    case 2: return leg2<T, 2>(p, s);
    case 3: return leg2<T, 3>(p, s);
    case 4: return leg2<T, 4>(p, s);
    case 5: return leg2<T, 5>(p, s);
    case 6: return leg2<T, 6>(p, s);
  }
  return cudaErrorInvalidValue;
}

// Spin-0 stage on the prepared T records (into d7) and, when phi is set, the
// potential's j <= 1 planes (into d7p) from the same recurrence.
cudaError_t launch_legendre_spin0(const tl_plan *p, int nder, bool phi, void *d7, void *d7p, cudaStream_t s) {
  if (p->precision == TL_FP64)
    return phi ? leg0_dispatch<double, true>(p, nder, d7, d7p, s) : leg0_dispatch<double, false>(p, nder, d7, d7p, s);
  return phi ? leg0_dispatch<float, true>(p, nder, d7, d7p, s) : leg0_dispatch<float, false>(p, nder, d7, d7p, s);
}

cudaError_t launch_legendre_spin2(const tl_plan *p, int nder, cudaStream_t s) {
  return p->precision == TL_FP64 ? leg2_dispatch<double>(p, nder, s) : leg2_dispatch<float>(p, nder, s);
}

}  // namespace tl
