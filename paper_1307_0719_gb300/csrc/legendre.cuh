// Legendre stage: per (ring, m), the theta-derivatives of the m-th Fourier
// coefficient of a field,
//     F^{j}_m(theta_r) = sum_l a_lm d^j/dtheta^j  s_lambda_lm(theta_r),   j <= NDER,
// computed by running the three-term recurrence in l on the fly and contracting
// it against the coefficients as it goes (Naess & Louis 2013, Sec. II.B: the
// derivative maps of Eq. 4; the paper obtains them by repeated SHTs).
//
// Recurrence (Wigner d-functions, spin s, fixed m):
//   lam_{l+1} = alpha_{l+1} (cos th + m s/(l(l+1))) lam_l - beta_{l+1} lam_{l-1},
//   alpha_L = sqrt((4L^2-1) L^2 / ((L^2-m^2)(L^2-s^2))),  beta_{l+1} = alpha_{l+1}/alpha_l.
// Its theta-dependence is only through cos(theta), so differentiating it j times
// with Leibniz's rule gives the derivative recurrence
//   lam^(j)_{l+1} = alpha_{l+1} [ X lam^(j)_l + sum_{i=1}^{j} C(j,i) cos^(i)(th) lam^(j-i)_l ]
//                   - beta_{l+1} lam^(j)_{l-1},       cos^(i)(th) = cos(th + i pi/2),
// which is exact and regular at every ring. Derivatives are carried divided by
// L^j (L = lmax+1) so that all orders share one floating-point range.
//
// Normalisation: mu_l = lam_l / k_l with k_{l+1} = beta_{l+1} k_{l-1}, so that
//   mu_{l+1} = A_{l+1} X mu_l - mu_{l-1},   A_{l+1} = alpha_{l+1} k_l / k_{l+1}.
// k_{l0} = 1 and k_{l0+1} is chosen so that the even and odd chains of k meet
// (k_{l+1}/k_l -> 1): then A_l -> 2 smoothly instead of alternating about 2, and
// the tables hold A - 2 (computed in double) so that A X - 2 keeps its precision.
//
// Two forms of the step. The double kernels run it as written (plain form). The
// float kernels run the difference form: with sg = sign(cos th), w = 1 - |cos th|
// and the state (mu_l, d_l = mu_l - sg mu_{l-1}),
//   c = Q - A w,  Q = (A - 2) + sg A m s/(l(l+1))        [= sg A (X + ms/(l(l+1))) - 2]
//   d_{l+1} = sg (c mu_l + d_l) + A sum_i C(j,i) cos^(i)(th) mu^(j-i)_l,
//   mu_{l+1} = sg mu_l + d_{l+1}.
// Near the poles A X - 2 is a small difference of numbers near 2, and float
// values of cos th and of A would each move it by ~1e-7, a large part of theta^2
// on the polar rings; the plain float step also amplifies its own rounding there
// (the two roots of the step meet at 1). The difference form uses w and A - 2,
// each exact to float precision, and its rounding of mu moves the state along the
// slowly varying solution (the idea of Reinsch's modification of the Goertzel
// recurrence), which keeps float results near 1e-6 on every ring.
//
// Seeds lam_{l0,m}, l0 = max(m,|s|), are N sin^a(th/2) cos^b(th/2); their
// logarithm and their theta-derivatives (via d^k/dth^k of ln sin(th/2) and
// ln cos(th/2), tabulated per ring) are formed in double precision. Values are
// held as mantissa * 2^(SB*sc) with an integer scale sc <= 0; a term contributes
// only once sc has climbed to 0, i.e. once the function is representable.
#pragma once

#include "common.cuh"

namespace tl {

template <typename T> struct RealTraits;
template <> struct RealTraits<float> {
  typedef float2 T2;
  typedef float4 T4;
  static constexpr double H = 32.0;    // rescale when |mantissa| > 2^H
  static constexpr int SB = 64;        // one scale step = 2^SB
  static constexpr float THR = 0x1p32f;     // 2^H
  static constexpr float STEP = 0x1p-64f;   // 2^-SB
};
template <> struct RealTraits<double> {
  typedef double2 T2;
  typedef double4 T4;
  static constexpr double H = 200.0;
  static constexpr int SB = 400;
  static constexpr double THR = 0x1p200;
  static constexpr double STEP = 0x1p-400;
};

// Coefficient record of the spin-0 stage at index idx(l, m): the coefficient
// times k_l, the factor A_{l+1} of the normalised step l -> l+1 and Q = A_{l+1} - 2.
template <typename T> struct __align__(4 * sizeof(T)) Rec0 {
  T re, im, A, Q;
};
// Spin-2 stage: k_l (E + iB), k_l (-1)^(l+m) (E - iB), A_{l+1}, C = m s/(l(l+1)) and
// the difference-form factors Qn = (A - 2) + A C (rings with cos th >= 0) and
// Qs = (A - 2) - A C (cos th < 0).
template <typename T> struct __align__(4 * sizeof(T)) Rec2 {
  T c1r, c1i, c2r, c2i;
  T A, cterm, Qn, Qs;
};

// ---------------------------------------------------------------------------
// recurrence pieces shared by the forward and adjoint Legendre kernels

// Binomial coefficient for small arguments; a plain loop, so that with the
// unrolled (constant) arguments of the kernels below it folds to a constant.
__host__ __device__ __forceinline__ constexpr int binom(int n, int k) {
  int r = 1;
  for (int t = 1; t <= k; ++t) r = r * (n - k + t) / t;
  return r;
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
  const double mant = sign * exp2(E - (double)RT::SB * s0);
  // d^j/dth^j f = f * B_j with B_{j+1} = sum_i C(j,i) g_{i+1} B_{j-i},
  // g_k = d^k/dth^k ln f = a d^k ln sin(th/2) + b d^k ln cos(th/2)
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

// Seed of the spin-0 recurrence at l0 = m: N_m sin^m(th/2) cos^m(th/2) (-1)^m.
template <typename T, int NDER>
__device__ __forceinline__ void seed_spin0(const RingTable &rt, const double *__restrict__ lnorm0, int r, int m,
                                           double invL, T (&cur)[NDER + 1], int &sc) {
  const double E = lnorm0[m] + (double)m * (rt.log2_sh[r] + rt.log2_ch[r]);
  seed_values<T, NDER>(rt, r, E, (double)m, (double)m, (m & 1) ? -1.0 : 1.0, invL, cur, sc);
}

// Seed of the spin-2 recurrence at l0 = max(m, 2); returns l0. For m >= 2 the
// seed is N_m sqrt(m(m-1)/((m+1)(m+2))) sin^(m+2)(th/2) cos^(m-2)(th/2); for
// m < 2, sqrt(5/4pi) sqrt(C(4, 2+m)) sin^(2+m)(th/2) cos^(2-m)(th/2); sign (-1)^m.
template <typename T, int NDER>
__device__ __forceinline__ int seed_spin2(const RingTable &rt, const double *__restrict__ lnorm0, int r, int m,
                                          double invL, T (&cur)[NDER + 1], int &sc) {
  const double lsh = rt.log2_sh[r], lch = rt.log2_ch[r];
  double E, ea, eb;
  int l0;
  if (m >= 2) {
    l0 = m;
    const double md = (double)m;
    E = lnorm0[m] + 0.5 * log2(md * (md - 1.0) / ((md + 1.0) * (md + 2.0))) + (md + 2.0) * lsh + (md - 2.0) * lch;
    ea = md + 2.0;
    eb = md - 2.0;
  } else {
    l0 = 2;
    const double c4 = (m == 0) ? 6.0 : 4.0;  // C(4, 2+m)
    E = log2(sqrt(5.0 / (4.0 * 3.14159265358979323846)) * sqrt(c4)) + (2.0 + m) * lsh + (2.0 - m) * lch;
    ea = 2.0 + m;
    eb = 2.0 - m;
  }
  seed_values<T, NDER>(rt, r, E, ea, eb, (m & 1) ? -1.0 : 1.0, invL, cur, sc);
  return l0;
}

// Leibniz coefficients e[j][i] = C(j, i) cos^(i)(theta) / L^i, i = 1..j, once per thread.
template <typename T, int NDER> struct Leib {
  T e[NDER + 1][NDER + 1];
};
template <typename T, int NDER>
__device__ __forceinline__ void leibniz_coefs(double x, double st, double invL, Leib<T, NDER> &L) {
  double p = 1.0, dc[NDER + 1];
#pragma unroll
  for (int i = 0; i <= NDER; ++i) {
    const double v = (i % 4 == 0) ? x : (i % 4 == 1) ? -st : (i % 4 == 2) ? -x : st;
    dc[i] = v * p;
    p *= invL;
  }
#pragma unroll
  for (int j = 0; j <= NDER; ++j)
#pragma unroll
    for (int i = 0; i <= NDER; ++i) L.e[j][i] = (i >= 1 && i <= j) ? (T)(binom(j, i) * dc[i]) : (T)0;
}

// Plain form, in place: old (mu_{l-1}) becomes mu_{l+1} from cur (mu_l):
//   old^(j) = A (X cur^(j) + sum_{i>=1} e[j][i] cur^(j-i)) - old^(j)
template <typename T, int NDER>
__device__ __forceinline__ void step_into(T (&old)[NDER + 1], const T (&cur)[NDER + 1], const Leib<T, NDER> &L,
                                          T X, T A) {
#pragma unroll
  for (int j = NDER; j >= 0; --j) {
    T acc = X * cur[j];
#pragma unroll
    for (int i = 1; i <= j; ++i) acc = fma(L.e[j][i], cur[j - i], acc);
    old[j] = fma(A, acc, -old[j]);
  }
}

// Difference form (SG = sign of cos th), in place: (v, d) = (mu_l, mu_l - SG mu_{l-1})
// become (mu_{l+1}, mu_{l+1} - SG mu_l); w = 1 - |cos th|, Q = Qn or Qs of the record.
template <typename T, int NDER, int SG>
__device__ __forceinline__ void step_diff(T (&v)[NDER + 1], T (&d)[NDER + 1], const Leib<T, NDER> &L, T w, T A,
                                          T Q) {
  const T c = fma(-A, w, Q);
#pragma unroll
  for (int j = NDER; j >= 0; --j) {
    T t = fma(c, v[j], d[j]);
    if (SG < 0) t = -t;
    if (j >= 1) {
      T acc = L.e[j][1] * v[j - 1];
#pragma unroll
      for (int i = 2; i <= j; ++i) acc = fma(L.e[j][i], v[j - i], acc);
      t = fma(A, acc, t);
    }
    d[j] = t;
    v[j] = (SG > 0) ? v[j] + t : t - v[j];
  }
}

// One step of either form for a T-typed kernel whose current values are in v:
// float runs the difference form (aux = d), double the plain form (aux = mu_{l-1},
// the new value rotated into v). X = cos th + C (plain), w, A, Q (difference).
template <typename T, int NDER, int SG>
__device__ __forceinline__ void rec_step(T (&aux)[NDER + 1], T (&v)[NDER + 1], const Leib<T, NDER> &L, T X, T w,
                                         T A, T Q) {
  if constexpr (sizeof(T) == 4) {
    step_diff<T, NDER, SG>(v, aux, L, w, A, Q);
  } else {
    step_into<T, NDER>(aux, v, L, X, A);
#pragma unroll
    for (int j = 0; j <= NDER; ++j) {
      const T t = aux[j];
      aux[j] = v[j];
      v[j] = t;
    }
  }
}

// State at l0 from the seed values in v: the plain form's mu_{l0-1} = 0, the
// difference form's d = mu_{l0} - SG * 0.
template <typename T, int NDER>
__device__ __forceinline__ void rec_init(T (&aux)[NDER + 1], const T (&v)[NDER + 1]) {
#pragma unroll
  for (int j = 0; j <= NDER; ++j) aux[j] = (sizeof(T) == 4) ? v[j] : (T)0;
}

// Exponent rescaling while the values are below the representable range.
template <typename T, int NDER>
__device__ __forceinline__ void rescale(T (&a)[NDER + 1], T (&b)[NDER + 1], const T lead, int &sc) {
  typedef RealTraits<T> RT;
  if (sc < 0 && fabs(lead) > RT::THR) {
#pragma unroll
    for (int j = 0; j <= NDER; ++j) {
      a[j] *= RT::STEP;
      b[j] *= RT::STEP;
    }
    ++sc;
  }
}

}  // namespace tl
