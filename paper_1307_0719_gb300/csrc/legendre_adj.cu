// Adjoint of the Legendre stage: from gradients with respect to the per-ring
// Fourier coefficients, Fbar^j_m(theta_r) (planes [j][ring][m], in the same
// normalised units as the forward planes: derivative order j carried over L^j),
// to gradients with respect to the coefficients a_lm,
//     abar_lm = k_l sum_r sum_j mu^(j)_lm(theta_r) G_lm(r, j),
// with the same on-the-fly recurrence (mu = lambda / k_l, see legendre.cu) and
// the transposed contraction (Naess & Louis 2013, Sec. II.B: the derivative maps
// of Eq. 4, here differentiated in reverse). Gradients follow the convention
// dL/dRe + i dL/dIm, so a complex coefficient c in F = c a contributes conj(c) Fbar.
//
// Spin 0 (one thread per north ring): with mu^(j)(pi - th) = (-1)^(l+m+j) mu^(j)(th),
//     G = Fbar_N + (-1)^(l+m+j) Fbar_S    (Fbar_S = 0 on the equator).
// Spin 2 (one thread per ring, north and mirror): the forward planes are
//     F^Q = -(S1 + (-1)^j S2')/2,  F^U = i (S1 - (-1)^j S2')/2,
//     S1 = sum_l k (E + iB) mu,  S2 = sum_l (-1)^(l+m) k (E - iB) mu  (' = mirror ring),
// so  S1bar(r) = -(Fbar^Q(r) + i Fbar^U(r))/2,  S2bar(r) = (-1)^j (-Fbar^Q(r') + i Fbar^U(r'))/2,
//     Ebar = k sum mu (S1bar + (-1)^(l+m) S2bar),  Bbar = -i k sum mu (S1bar - (-1)^(l+m) S2bar).
//
// Reduction over rings. Every l needs a sum over all rings; each thread writes
// its V contributions for a window of W consecutive l into shared memory, the
// block sums the window (a few adjacent lanes per output, combined by lane
// shuffles) and adds it to the double accumulators with one atomic per
// (l, component) and block. k_l is applied afterwards.
#include <math.h>

#include "legendre.cuh"

namespace tl {

// Outputs (l, component) per window: 64 for float, 32 for double, so that the
// window [128 threads][WV + 1] stays within 34 KB of static shared memory.
template <typename T> struct AdjWin {
  static constexpr int WV = 256 / (int)sizeof(T);
};

// Sum of the window [lb, lb + nl) over the block's NT threads into acc.
// win: [NT][WV + 1]; output o is summed by NP = NT / WV adjacent lanes.
template <typename T, int NT, int WV, int V>
__device__ __forceinline__ void flush_window(T (*win)[WV + 1], int nl, long long idx0, double *acc0, double *acc1) {
  constexpr int NP = NT / WV;
  static_assert(NP * WV == NT && (NP & (NP - 1)) == 0 && NP <= 32, "window split");
  __syncthreads();
  const int t = threadIdx.x;
  const int o = t / NP, part = t % NP;
  T sum = (T)0;
#pragma unroll 8
  for (int i = part; i < NT; i += NP) sum += win[i][o];
#pragma unroll
  for (int d = 1; d < NP; d <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
  const int li = o / V, c = o - (o / V) * V;
  if (part == 0 && li < nl) {
    // components: 0, 1 -> acc0 (re, im); 2, 3 -> acc1 (re, im)
    double *a = (c < 2) ? acc0 : acc1;
    if (a) atomicAdd(a + 2 * (idx0 + li) + (c & 1), (double)sum);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// spin 0: T with derivative orders j <= nder_T and, with PHI, the lensing
// potential's j <= 1 planes, both against the same recurrence.

template <typename T, int NDER, bool PHI>
__global__ void __launch_bounds__(128) legendre_adj0_kernel(RingTable rt, const double *__restrict__ lnorm0,
                                                            int nside, int lmax, int mmax, int nrings, int nder_T,
                                                            const typename RealTraits<T>::T2 *__restrict__ tab,
                                                            const typename RealTraits<T>::T2 *__restrict__ FT,
                                                            const typename RealTraits<T>::T2 *__restrict__ FP,
                                                            double *__restrict__ accT, double *__restrict__ accP) {
  typedef typename RealTraits<T>::T2 T2;
  constexpr int NT = 128, WV = AdjWin<T>::WV, V = PHI ? 4 : 2, W = WV / V;
  __shared__ T win[NT][WV + 1];
  const int m = blockIdx.y;
  const int tid = threadIdx.x;
  const int rn = blockIdx.x * NT + tid;
  const bool active = rn < 2 * nside && m <= mmax;
  const int r = active ? rn : 0;
  const int rs = nrings - 1 - r;
  const double invL = 1.0 / (double)(lmax + 1);
  const size_t ld = (size_t)(mmax + 1);
  const int mm = m <= mmax ? m : mmax;

  // G+ (even l - m) and G- (odd l - m) per derivative order
  T gpr[NDER + 1], gpi[NDER + 1], gmr[NDER + 1], gmi[NDER + 1];
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    T2 fn = {(T)0, (T)0}, fs = {(T)0, (T)0};
    if (active && j <= nder_T) {
      fn = FT[((size_t)j * nrings + r) * ld + mm];
      if (rs != r) fs = FT[((size_t)j * nrings + rs) * ld + mm];
    }
    const T sg = (j & 1) ? (T)-1 : (T)1;
    gpr[j] = fn.x + sg * fs.x;
    gpi[j] = fn.y + sg * fs.y;
    gmr[j] = fn.x - sg * fs.x;
    gmi[j] = fn.y - sg * fs.y;
  }
  T hpr[2], hpi[2], hmr[2], hmi[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    T2 fn = {(T)0, (T)0}, fs = {(T)0, (T)0};
    if (PHI && active) {
      fn = FP[((size_t)j * nrings + r) * ld + mm];
      if (rs != r) fs = FP[((size_t)j * nrings + rs) * ld + mm];
    }
    const T sg = (j & 1) ? (T)-1 : (T)1;
    hpr[j] = fn.x + sg * fs.x;
    hpi[j] = fn.y + sg * fs.y;
    hmr[j] = fn.x - sg * fs.x;
    hmi[j] = fn.y - sg * fs.y;
  }

  const double x = rt.z[r], st = rt.sint[r];
  Leib<T, NDER> LC;
  leibniz_coefs<T, NDER>(x, st, invL, LC);
  T a[NDER + 1], b[NDER + 1];  // b = mu_l; a = d_l (float) or mu_{l-1} (double)
  int sc;
  seed_spin0<T, NDER>(rt, lnorm0, r, m, invL, b, sc);
  rec_init<T, NDER>(a, b);

  const long long base = (long long)m * (2 * lmax + 1 - m) / 2;
  const T2 *tm = tab + base;  // {k_l, A_{l+1} - 2}
  const T X = (T)x, w = (T)rt.omza[r];
  int lb = m;  // first l of the current window
  for (int l = m;; l += 2) {
    // ---- even l - m
    {
      const int li = l - lb;
      T cr = (T)0, ci = (T)0, pr = (T)0, pi = (T)0;
      if (sc == 0) {
#pragma unroll
        for (int j = 0; j <= NDER; ++j) {
          cr = fma(b[j], gpr[j], cr);
          ci = fma(b[j], gpi[j], ci);
        }
        if (PHI) {
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            pr = fma(b[j], hpr[j], pr);
            pi = fma(b[j], hpi[j], pi);
          }
        }
      }
      win[tid][li * V + 0] = cr;
      win[tid][li * V + 1] = ci;
      if (PHI) {
        win[tid][li * V + 2] = pr;
        win[tid][li * V + 3] = pi;
      }
      if (l == lmax || li == W - 1) {
        flush_window<T, NT, WV, V>(win, li + 1, base + lb, accT, PHI ? accP : nullptr);
        lb += W;
      }
      if (l == lmax) break;
      const T Q = tm[l].y;
      rec_step<T, NDER, 1>(a, b, LC, X, w, (T)2 + Q, Q);
      rescale<T, NDER>(a, b, b[0], sc);
    }
    // ---- odd l - m
    {
      const int li = l + 1 - lb;
      T cr = (T)0, ci = (T)0, pr = (T)0, pi = (T)0;
      if (sc == 0) {
#pragma unroll
        for (int j = 0; j <= NDER; ++j) {
          cr = fma(b[j], gmr[j], cr);
          ci = fma(b[j], gmi[j], ci);
        }
        if (PHI) {
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            pr = fma(b[j], hmr[j], pr);
            pi = fma(b[j], hmi[j], pi);
          }
        }
      }
      win[tid][li * V + 0] = cr;
      win[tid][li * V + 1] = ci;
      if (PHI) {
        win[tid][li * V + 2] = pr;
        win[tid][li * V + 3] = pi;
      }
      if (l + 1 == lmax || li == W - 1) {
        flush_window<T, NT, WV, V>(win, li + 1, base + lb, accT, PHI ? accP : nullptr);
        lb += W;
      }
      if (l + 1 == lmax) break;
      const T Q = tm[l + 1].y;
      rec_step<T, NDER, 1>(a, b, LC, X, w, (T)2 + Q, Q);
      rescale<T, NDER>(a, b, b[0], sc);
    }
  }
}

// ---------------------------------------------------------------------------
// spin 2: block = 64 north rings and their 64 mirrors (one thread each).

// Recurrence of one ring (SG = sign cos th) with the transposed contraction into
// the block's l windows; U1 = S1bar + S2bar (even l + m), U2 = S1bar - S2bar (odd).
template <typename T, int NDER, int SG, int WV>
__device__ __forceinline__ void adj2_sweep(const Rec2<T> *__restrict__ rm, int l0, int m, int lmax, long long base,
                                           const Leib<T, NDER> &LC, T X, T w, T (&a)[NDER + 1], T (&b)[NDER + 1],
                                           int &sc, const T (&u1r)[NDER + 1], const T (&u1i)[NDER + 1],
                                           const T (&u2r)[NDER + 1], const T (&u2i)[NDER + 1],
                                           T (*win)[WV + 1], double *accE, double *accB) {
  constexpr int NT = 128, V = 4, W = WV / V;
  const int t = threadIdx.x;
  int lb = l0;
  const int par0 = (l0 + m) & 1;  // parity of l + m at l0
  for (int l = l0;; l += 2) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int ll = l + half;
      const int li = ll - lb;
      const bool even = ((par0 + half) & 1) == 0;
      T er = (T)0, ei = (T)0, fr = (T)0, fi = (T)0;
      if (sc == 0) {
#pragma unroll
        for (int j = 0; j <= NDER; ++j) {
          const T p1r = even ? u1r[j] : u2r[j], p1i = even ? u1i[j] : u2i[j];
          const T p2r = even ? u2r[j] : u1r[j], p2i = even ? u2i[j] : u1i[j];
          er = fma(b[j], p1r, er);
          ei = fma(b[j], p1i, ei);
          fr = fma(b[j], p2r, fr);
          fi = fma(b[j], p2i, fi);
        }
      }
      win[t][li * V + 0] = er;
      win[t][li * V + 1] = ei;
      win[t][li * V + 2] = fr;
      win[t][li * V + 3] = fi;
      if (ll == lmax || li == W - 1) {
        flush_window<T, NT, WV, V>(win, li + 1, base + lb, accE, accB);
        lb += W;
      }
      if (ll == lmax) return;
      const Rec2<T> c = rm[ll];
      rec_step<T, NDER, SG>(a, b, LC, X + c.cterm, w, c.A, SG > 0 ? c.Qn : c.Qs);
      rescale<T, NDER>(a, b, b[0], sc);
    }
    if (l + 1 >= lmax) return;
  }
}

template <typename T, int NDER>
__global__ void __launch_bounds__(128) legendre_adj2_kernel(RingTable rt, const double *__restrict__ lnorm0,
                                                            int nside, int lmax, int mmax, int nrings,
                                                            const Rec2<T> *__restrict__ rec,
                                                            const typename RealTraits<T>::T2 *__restrict__ FQ,
                                                            const typename RealTraits<T>::T2 *__restrict__ FU,
                                                            double *__restrict__ accE, double *__restrict__ accB) {
  typedef typename RealTraits<T>::T2 T2;
  constexpr int NT = 128, RP = 64, WV = AdjWin<T>::WV, V = 4, W = WV / V;
  __shared__ T win[NT][WV + 1];
  const int m = blockIdx.y;
  const int t = threadIdx.x;
  const int rn = blockIdx.x * RP + (t % RP);
  const bool mirror = t >= RP;
  const bool equator = rn == nrings - 1 - rn;
  // the equator ring is its own mirror: its north thread carries both terms
  const bool active = rn < 2 * nside && m <= mmax && !(mirror && equator);
  const int r = rn < 2 * nside ? (mirror ? nrings - 1 - rn : rn) : 0;
  const int rp = nrings - 1 - r;  // partner (mirror) ring
  const double invL = 1.0 / (double)(lmax + 1);
  const size_t ld = (size_t)(mmax + 1);
  const int mm = m <= mmax ? m : mmax;

  // U1 = S1bar + S2bar (even l + m), U2 = S1bar - S2bar (odd l + m)
  T u1r[NDER + 1], u1i[NDER + 1], u2r[NDER + 1], u2i[NDER + 1];
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    T2 q = {(T)0, (T)0}, u = {(T)0, (T)0}, qp = {(T)0, (T)0}, up = {(T)0, (T)0};
    if (active) {
      q = FQ[((size_t)j * nrings + r) * ld + mm];
      u = FU[((size_t)j * nrings + r) * ld + mm];
      qp = FQ[((size_t)j * nrings + rp) * ld + mm];
      up = FU[((size_t)j * nrings + rp) * ld + mm];
    }
    const T h = (T)0.5, sg = (j & 1) ? (T)-0.5 : (T)0.5;
    // S1bar = -(q + i u)/2
    const T s1r = -h * (q.x - u.y), s1i = -h * (q.y + u.x);
    // S2bar = (-1)^j (-qp + i up)/2
    const T s2r = sg * (-qp.x - up.y), s2i = sg * (-qp.y + up.x);
    u1r[j] = s1r + s2r;
    u1i[j] = s1i + s2i;
    u2r[j] = s1r - s2r;
    u2i[j] = s1i - s2i;
  }

  const double x = rt.z[r], st = rt.sint[r];
  Leib<T, NDER> LC;
  leibniz_coefs<T, NDER>(x, st, invL, LC);
  T a[NDER + 1], b[NDER + 1];  // b = mu_l; a = d_l (float) or mu_{l-1} (double)
  int sc;
  const int l0 = seed_spin2<T, NDER>(rt, lnorm0, r, m, invL, b, sc);
  rec_init<T, NDER>(a, b);
  if (l0 > lmax) return;  // uniform over the block

  const long long base = (long long)m * (2 * lmax + 1 - m) / 2;
  const Rec2<T> *rm = rec + base;
  const T X = (T)x, w = (T)rt.omza[r];
  // mirror threads (cos th < 0) are warps 2 and 3; the window flushes inside keep
  // every thread of the block in step, so both branches run the same l sequence
  if (mirror)
    adj2_sweep<T, NDER, -1, WV>(rm, l0, m, lmax, base, LC, X, w, a, b, sc, u1r, u1i, u2r, u2i, win, accE, accB);
  else
    adj2_sweep<T, NDER, 1, WV>(rm, l0, m, lmax, base, LC, X, w, a, b, sc, u1r, u1i, u2r, u2i, win, accE, accB);
}

// Final scaling: abar = k_l acc; B's accumulator holds f with Bbar = -i k f;
// m = 0 coefficients are real in the forward map, so their imaginary gradient is 0.
template <typename T>
__global__ void adj_finish_kernel(int lmax, const typename RealTraits<T>::T2 *__restrict__ tab0,
                                  const typename RealTraits<T>::T2 *__restrict__ tab2, double *__restrict__ gT,
                                  double *__restrict__ gP, double *__restrict__ gE, double *__restrict__ gB) {
  const int m = blockIdx.y;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  const long long idx = (long long)m * (2 * lmax + 1 - m) / 2 + l;
  const double k0 = (double)tab0[idx].x;
  if (gT) {
    gT[2 * idx] *= k0;
    gT[2 * idx + 1] = (m == 0) ? 0.0 : gT[2 * idx + 1] * k0;
  }
  if (gP) {
    gP[2 * idx] *= k0;
    gP[2 * idx + 1] = (m == 0) ? 0.0 : gP[2 * idx + 1] * k0;
  }
  if (tab2) {
    const double k2 = (double)tab2[idx].x;  // 0 for l < 2
    if (gE) {
      gE[2 * idx] *= k2;
      gE[2 * idx + 1] = (m == 0) ? 0.0 : gE[2 * idx + 1] * k2;
    }
    if (gB) {
      const double fr = gB[2 * idx], fi = gB[2 * idx + 1];
      gB[2 * idx] = k2 * fi;
      gB[2 * idx + 1] = (m == 0) ? 0.0 : -k2 * fr;
    }
  }
}

// ---------------------------------------------------------------------------
// launchers

template <typename T, int NDER, bool PHI>
static cudaError_t adj0(const tl_plan *p, int nder_T, const void *FT, const void *FP, double *aT, double *aP,
                        cudaStream_t s) {
  typedef typename RealTraits<T>::T2 T2;
  dim3 grid((2 * p->nside + 127) / 128, p->mmax + 1);
  legendre_adj0_kernel<T, NDER, PHI><<<grid, 128, 0, s>>>(p->ring, p->lnorm0, p->nside, p->lmax, p->mmax,
                                                          p->nrings, nder_T, (const T2 *)p->tab0, (const T2 *)FT,
                                                          (const T2 *)FP, aT, aP);
  return cudaGetLastError();
}

template <typename T, bool PHI>
static cudaError_t adj0_dispatch(const tl_plan *p, int nder, int nder_T, const void *FT, const void *FP, double *aT,
                                 double *aP, cudaStream_t s) {
  switch (nder) {
    case 0: return PHI ? cudaErrorInvalidValue : adj0<T, 0, false>(p, nder_T, FT, FP, aT, aP, s);
    case 1: return adj0<T, 1, PHI>(p, nder_T, FT, FP, aT, aP, s);
    case 2: return adj0<T, 2, PHI>(p, nder_T, FT, FP, aT, aP, s);
    case 3: return adj0<T, 3, PHI>(p, nder_T, FT, FP, aT, aP, s);
    case 4: return adj0<T, 4, PHI>(p, nder_T, FT, FP, aT, aP, s);
    case 5: return adj0<T, 5, PHI>(p, nder_T, FT, FP, aT, aP, s);
    case 6: return adj0<T, 6, PHI>(p, nder_T, FT, FP, aT, aP, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_legendre_adj0(const tl_plan *p, int nder_T, const void *FT, const void *FP, double *aT,
                                 double *aP, cudaStream_t s) {
  const bool phi = FP && aP;
  const int nder = (phi && nder_T < 1) ? 1 : nder_T;
  if (p->precision == TL_FP64)
    return phi ? adj0_dispatch<double, true>(p, nder, nder_T, FT, FP, aT, aP, s)
               : adj0_dispatch<double, false>(p, nder, nder_T, FT, FP, aT, nullptr, s);
  return phi ? adj0_dispatch<float, true>(p, nder, nder_T, FT, FP, aT, aP, s)
             : adj0_dispatch<float, false>(p, nder, nder_T, FT, FP, aT, nullptr, s);
}

template <typename T, int NDER>
static cudaError_t adj2(const tl_plan *p, const void *FQ, const void *FU, double *aE, double *aB, cudaStream_t s) {
  typedef typename RealTraits<T>::T2 T2;
  dim3 grid((2 * p->nside + 63) / 64, p->mmax + 1);
  legendre_adj2_kernel<T, NDER><<<grid, 128, 0, s>>>(p->ring, p->lnorm0, p->nside, p->lmax, p->mmax, p->nrings,
                                                     (const Rec2<T> *)p->rec_QU, (const T2 *)FQ, (const T2 *)FU, aE,
                                                     aB);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t adj2_dispatch(const tl_plan *p, int nder, const void *FQ, const void *FU, double *aE, double *aB,
                                 cudaStream_t s) {
  switch (nder) {
    case 0: return adj2<T, 0>(p, FQ, FU, aE, aB, s);
    case 1: return adj2<T, 1>(p, FQ, FU, aE, aB, s);
    case 2: return adj2<T, 2>(p, FQ, FU, aE, aB, s);
    case 3: return adj2<T, 3>(p, FQ, FU, aE, aB, s);
    case 4: return adj2<T, 4>(p, FQ, FU, aE, aB, s);
    case 5: return adj2<T, 5>(p, FQ, FU, aE, aB, s);
    case 6: return adj2<T, 6>(p, FQ, FU, aE, aB, s);
  }
  return cudaErrorInvalidValue;
}

// Needs rec_QU prepared (its A_{l+1} and m s/(l(l+1)) fields are used).
cudaError_t launch_legendre_adj2(const tl_plan *p, int nder, const void *FQ, const void *FU, double *aE, double *aB,
                                 cudaStream_t s) {
  return p->precision == TL_FP64 ? adj2_dispatch<double>(p, nder, FQ, FU, aE, aB, s)
                                 : adj2_dispatch<float>(p, nder, FQ, FU, aE, aB, s);
}

template <typename T>
static cudaError_t finish_t(const tl_plan *p, double *gT, double *gP, double *gE, double *gB, cudaStream_t s) {
  typedef typename RealTraits<T>::T2 T2;
  dim3 grid((p->lmax + 1 + 127) / 128, p->lmax + 1);
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  adj_finish_kernel<T><<<grid, 128, 0, s>>>(p->lmax, (const T2 *)p->tab0, pol ? (const T2 *)p->tab2 : nullptr, gT,
                                            gP, gE, gB);
  return cudaGetLastError();
}

cudaError_t launch_adj_finish(const tl_plan *p, double *gT, double *gP, double *gE, double *gB, cudaStream_t s) {
  return p->precision == TL_FP64 ? finish_t<double>(p, gT, gP, gE, gB, s) : finish_t<float>(p, gT, gP, gE, gB, s);
}

}  // namespace tl
