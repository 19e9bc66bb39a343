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
// times k_l and the factor A_{l+1} of the normalised step l -> l+1.
template <typename T> struct __align__(4 * sizeof(T)) Rec0 {
  T re, im, A, pad;
};
// Spin-2 stage: k_l (E + iB), k_l (-1)^(l+m) (E - iB), A_{l+1} and m s/(l(l+1)).
template <typename T> struct __align__(4 * sizeof(T)) Rec2 {
  T c1r, c1i, c2r, c2i;
  T A, cterm, pad0, pad1;
};

}  // namespace tl
