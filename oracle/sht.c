/*
 * Oracle -- TEST INFRASTRUCTURE ONLY. Plain, slow, FP64 CPU reference for the
 * spherical-harmonic part of full-sky Taylor lensing (Naess & Louis 2013).
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may call it;
 * the GPU library never links or loads it, and it shares no code with it.
 *
 * What it computes (Sec. II.B, Eq. 4): for every iso-latitude ring theta and
 * every m >= 0, the theta-derivatives of order j <= nder of the m-th Fourier
 * coefficient of the unlensed fields,
 *
 *   F^{T,j}_m(theta) = sum_l T_lm  d^j/dtheta^j  0lambda_lm(theta)
 *   F^{Q,j}_m(theta) = -sum_l ( E_lm lam+^(j) + i B_lm lam-^(j) )
 *   F^{U,j}_m(theta) =  sum_l ( i E_lm lam-^(j) - B_lm lam+^(j) )
 *
 * with lam+- = (2lambda_lm +- -2lambda_lm)/2, i.e. Q +- iU = -sum (E +- iB) +-2Y_lm
 * (the HEALPix polarisation convention the paper inherits from healpy).
 *
 * Definitions used, written out plainly:
 *  - sY_lm(theta,phi) = slambda_lm(theta) e^{i m phi}, with the spin-raising
 *    operator  eth f = -(d_theta - s cot(theta) - m csc(theta)) f  and
 *    eth sY = sqrt((l-s)(l+s+1)) s+1Y,  bar-eth sY = -sqrt((l+s)(l-s+1)) s-1Y
 *    (Goldberg et al. 1967); spin 0 is the usual Y_lm with Condon-Shortley phase.
 *  - slambda_lm by the three-term recurrence in l of the Wigner d-functions,
 *      slam_{l+1} = alpha_{l+1} [ (cos theta + m s/(l(l+1))) slam_l - slam_{l-1}/alpha_l ],
 *      alpha_l   = sqrt( (4l^2-1) l^2 / ((l^2-m^2)(l^2-s^2)) ),
 *    started at l0 = max(m,|s|) from the closed-form d^{l0} seed.
 *  - theta-derivatives from the ladder identity d_theta = -(eth + bar-eth)/2,
 *    applied j times to the vector of spins s-j..s+j at fixed (l, m).
 * Values are carried as mantissa * 2^exponent so that seeds as small as
 * sin^m(theta) with m ~ 10^4 do not underflow; any final value below the
 * smallest double is returned as 0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ---- scaled numbers: value = v * 2^e ------------------------------------ */
typedef struct { double v; long e; } xnum;

static xnum xnorm(double v, long e) {
  xnum r;
  if (v == 0.0) { r.v = 0.0; r.e = 0; return r; }
  int k; r.v = frexp(v, &k); r.e = e + k;
  return r;
}

/* Seed slambda_{l0,m}(theta), l0 = max(m,|s|). Returns l0 and the scaled value. */
static int spin_seed(int m, int s, double theta, xnum *out) {
  int a = abs(s);
  double sh = sin(0.5 * theta), ch = cos(0.5 * theta);
  if (m >= a) {
    /* (-1)^m sqrt((2m+1)/4pi) sqrt(C(2m, m+s)) sin^{m+s}(t/2) cos^{m-s}(t/2)
       = (-1)^m sqrt((2m+1)/4pi) prod_k sqrt((2k-1)/(2k)) sin^m(t)
         * sqrt(C(2m,m+s)/C(2m,m)) * tan^s(t/2)                           */
    xnum x = xnorm(1.0, 0);
    double st = sin(theta);
    for (int k = 1; k <= m; ++k) {
      x = xnorm(x.v * sqrt((2.0 * k - 1.0) / (2.0 * k)) * st, x.e);
    }
    double ratio = 1.0; /* C(2m,m+|s|)/C(2m,m) = prod_{k=1}^{|s|} (m-|s|+k)/(m+k) */
    for (int k = 1; k <= a; ++k) ratio *= (double)(m - a + k) / (double)(m + k);
    double t = sh / ch, tp = 1.0;
    for (int k = 0; k < a; ++k) tp *= (s > 0 ? t : 1.0 / t);
    double pre = sqrt((2.0 * m + 1.0) / (4.0 * ORC_PI)) * sqrt(ratio) * tp;
    if (m & 1) pre = -pre;
    *out = xnorm(x.v * pre, x.e);
    return m;
  }
  /* |s| > m: l0 = |s| */
  double binom = 1.0; /* C(2a, a+m) */
  for (int k = 1; k <= a - m; ++k) binom *= (double)(a + m + k) / (double)k;
  double pre = sqrt((2.0 * a + 1.0) / (4.0 * ORC_PI)) * sqrt(binom);
  double val;
  if (s > 0) {
    val = pre * pow(sh, s + m) * pow(ch, s - m);
    if (m & 1) val = -val;
  } else {
    val = pre * pow(sh, a - m) * pow(ch, a + m);
    if (a & 1) val = -val;
  }
  *out = xnorm(val, 0);
  return a;
}

/* out[l] = slambda_lm(theta) for l = 0..lmax (zero below l0). */
void orc_spin_lambda(int lmax, int m, int s, double theta, double *out) {
  for (int l = 0; l <= lmax; ++l) out[l] = 0.0;
  xnum seed;
  int l0 = spin_seed(m, s, theta, &seed);
  if (l0 > lmax) return;
  double x = cos(theta);
  double mm = (double)m * m, ss = (double)s * s;
  double prev = 0.0, cur = seed.v;
  long e = seed.e;
  out[l0] = ldexp(cur, (int)(e < -4000 ? -4000 : e));
  double alpha_l = 0.0;
  for (int l = l0; l < lmax; ++l) {
    double L = l + 1.0;
    double alpha_n = sqrt((4.0 * L * L - 1.0) * L * L / ((L * L - mm) * (L * L - ss)));
    double c = (l == 0) ? 0.0 : (double)m * s / ((double)l * (l + 1.0));
    double nxt = alpha_n * ((x + c) * cur - (l > l0 ? prev / alpha_l : 0.0));
    prev = cur; cur = nxt; alpha_l = alpha_n;
    if (fabs(cur) > 0x1p+300) { cur = ldexp(cur, -300); prev = ldexp(prev, -300); e += 300; }
    out[l + 1] = ldexp(cur, (int)(e < -4000 ? -4000 : e));
  }
}

/* Ladder coefficients, zero where the neighbouring spin does not exist. */
static double kp(int l, int s) { /* eth: s -> s+1 */
  if (abs(s) > l || abs(s + 1) > l) return 0.0;
  return sqrt((double)(l - s) * (double)(l + s + 1));
}
static double km(int l, int s) { /* bar-eth: s -> s-1 (without its minus sign) */
  if (abs(s) > l || abs(s - 1) > l) return 0.0;
  return sqrt((double)(l + s) * (double)(l - s + 1));
}

/* out[j*(lmax+1)+l] = d^j/dtheta^j slambda_lm(theta), j = 0..nder. */
void orc_spin_lambda_derivs(int lmax, int m, int s, int nder, double theta, double *out) {
  int ns = 2 * nder + 1;
  double *base = (double *)malloc(sizeof(double) * ns * (lmax + 1));
  for (int t = 0; t < ns; ++t) orc_spin_lambda(lmax, m, s - nder + t, theta, base + (size_t)t * (lmax + 1));
  double v[64], w[64];
  for (int l = 0; l <= lmax; ++l) {
    for (int t = 0; t < ns; ++t) v[t] = base[(size_t)t * (lmax + 1) + l];
    out[l] = v[nder];
    for (int j = 1; j <= nder; ++j) {
      /* d_theta sY = -(eth sY + bar-eth sY)/2
                    = -(1/2) [ kp(l,s) s+1Y - km(l,s) s-1Y ]  */
      for (int t = j; t < ns - j; ++t) {
        int sp = s - nder + t;
        w[t] = -0.5 * (kp(l, sp) * v[t + 1] - km(l, sp) * v[t - 1]);
      }
      for (int t = j; t < ns - j; ++t) v[t] = w[t];
      out[(size_t)j * (lmax + 1) + l] = v[nder];
    }
  }
  free(base);
}

/*
 * Per-ring Fourier coefficients of the field derivatives.
 * alm_*: complex128 interleaved (re, im), triangular layout m(2lmax+1-m)/2 + l,
 *        any of them may be NULL (treated as zero; T NULL => FT untouched,
 *        E and B both NULL => FQ, FU untouched).
 * F*:    [nth][nder+1][mmax+1] complex128 interleaved.
 */
void orc_ring_coeffs(int lmax, int mmax, int nder, int nth, const double *theta,
                     const double *alm_T, const double *alm_E, const double *alm_B,
                     double *FT, double *FQ, double *FU, int nthreads) {
  int pol = (alm_E != NULL || alm_B != NULL);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
  {
    size_t L1 = (size_t)lmax + 1;
    double *d0 = (double *)malloc(sizeof(double) * (nder + 1) * L1);
    double *dp = (double *)malloc(sizeof(double) * (nder + 1) * L1);
    double *dm = (double *)malloc(sizeof(double) * (nder + 1) * L1);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int r = 0; r < nth; ++r) {
      for (int m = 0; m <= mmax; ++m) {
        size_t base = (size_t)m * (2 * lmax + 1 - m) / 2;
        if (alm_T) orc_spin_lambda_derivs(lmax, m, 0, nder, theta[r], d0);
        if (pol) {
          orc_spin_lambda_derivs(lmax, m, 2, nder, theta[r], dp);
          orc_spin_lambda_derivs(lmax, m, -2, nder, theta[r], dm);
        }
        for (int j = 0; j <= nder; ++j) {
          size_t o = (((size_t)r * (nder + 1) + j) * (mmax + 1) + m) * 2;
          if (alm_T) {
            double re = 0.0, im = 0.0;
            for (int l = m; l <= lmax; ++l) {
              double lam = d0[j * L1 + l];
              re += alm_T[2 * (base + l)] * lam;
              im += alm_T[2 * (base + l) + 1] * lam;
            }
            FT[o] = re; FT[o + 1] = im;
          }
          if (pol) {
            double qre = 0, qim = 0, ure = 0, uim = 0;
            for (int l = (m > 2 ? m : 2); l <= lmax; ++l) {
              double lp = 0.5 * (dp[j * L1 + l] + dm[j * L1 + l]);
              double lmn = 0.5 * (dp[j * L1 + l] - dm[j * L1 + l]);
              double er = alm_E ? alm_E[2 * (base + l)] : 0.0, ei = alm_E ? alm_E[2 * (base + l) + 1] : 0.0;
              double br = alm_B ? alm_B[2 * (base + l)] : 0.0, bi = alm_B ? alm_B[2 * (base + l) + 1] : 0.0;
              /* FQ = -(E lp + i B lmn) ; FU = i E lmn - B lp */
              qre += -(er * lp) + bi * lmn;
              qim += -(ei * lp) - br * lmn;
              ure += -ei * lmn - br * lp;
              uim += er * lmn - bi * lp;
            }
            FQ[o] = qre; FQ[o + 1] = qim;
            FU[o] = ure; FU[o + 1] = uim;
          }
        }
      }
    }
    free(d0); free(dp); free(dm);
  }
}

/*
 * Direct evaluation at arbitrary points (brute force and sampled checks):
 * value of the order-(j,k) derivative of T, Q, U at (theta_p, phi_p) from the
 * ring coefficients of a single point, summing the Fourier series directly:
 *   D(theta, phi) = Re[ F_0 + 2 sum_{m>=1} (i m)^k F_m e^{i m phi} ].
 * F: [npts][nder+1][mmax+1] complex (one "ring" per point, as produced by
 * orc_ring_coeffs with theta = theta_p). out: [npts] for the chosen (j, k).
 */
void orc_point_sum(int mmax, int nder, int npts, const double *F, const double *phi,
                   int j, int k, double *out, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
  for (int p = 0; p < npts; ++p) {
    double acc = 0.0;
    for (int m = 0; m <= mmax; ++m) {
      size_t o = (((size_t)p * (nder + 1) + j) * (mmax + 1) + m) * 2;
      double fr = F[o], fi = F[o + 1];
      /* (i m)^k */
      double pr = 1.0, pi_ = 0.0;
      for (int t = 0; t < k; ++t) { double nr = -pi_ * m, ni = pr * m; pr = nr; pi_ = ni; }
      double gr = fr * pr - fi * pi_, gi = fr * pi_ + fi * pr;
      double c = cos(m * phi[p]), s = sin(m * phi[p]);
      double term = gr * c - gi * s;
      acc += (m == 0 ? 1.0 : 2.0) * term;
    }
    out[p] = acc;
  }
}

/*
 * Transpose of orc_ring_coeffs: given per-ring coefficient gradients
 * Fb*[r][j][m] (complex, dL/dRe + i dL/dIm of F^{s,j}_m(theta_r)), accumulate the
 * coefficient gradients (dL/dRe + i dL/dIm of the stored a_lm, m >= 0):
 *   Tbar_lm = sum_{r,j} d^j 0lambda_lm(theta_r) FbT^j_m(r)
 *   Ebar_lm = sum_{r,j} [ -lam+^(j) FbQ^j_m - i lam-^(j) FbU^j_m ]
 *   Bbar_lm = sum_{r,j} [  i lam-^(j) FbQ^j_m - lam+^(j) FbU^j_m ]
 * (for F = kappa a with complex kappa the gradient of a is conj(kappa) Fbar).
 * The m = 0 imaginary parts, which the forward map ignores, are returned as 0.
 * Parallel over m. Outputs are overwritten.
 */
void orc_ring_adjoint(int lmax, int mmax, int nder, int nth, const double *theta, const double *FbT,
                      const double *FbQ, const double *FbU, double *aT, double *aE, double *aB, int nthreads) {
  size_t na = (size_t)(lmax + 1) * (lmax + 2) / 2;
  if (aT) memset(aT, 0, sizeof(double) * 2 * na);
  if (aE) memset(aE, 0, sizeof(double) * 2 * na);
  if (aB) memset(aB, 0, sizeof(double) * 2 * na);
  int pol = (FbQ != NULL);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
  {
    size_t L1 = (size_t)lmax + 1;
    double *d0 = (double *)malloc(sizeof(double) * (nder + 1) * L1);
    double *dp = (double *)malloc(sizeof(double) * (nder + 1) * L1);
    double *dm = (double *)malloc(sizeof(double) * (nder + 1) * L1);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int m = 0; m <= mmax; ++m) {
      size_t base = (size_t)m * (2 * lmax + 1 - m) / 2;
      for (int r = 0; r < nth; ++r) {
        if (FbT) orc_spin_lambda_derivs(lmax, m, 0, nder, theta[r], d0);
        if (pol) {
          orc_spin_lambda_derivs(lmax, m, 2, nder, theta[r], dp);
          orc_spin_lambda_derivs(lmax, m, -2, nder, theta[r], dm);
        }
        for (int j = 0; j <= nder; ++j) {
          size_t o = (((size_t)r * (nder + 1) + j) * (mmax + 1) + m) * 2;
          if (FbT) {
            double fr = FbT[o], fi = FbT[o + 1];
            for (int l = m; l <= lmax; ++l) {
              double lam = d0[j * L1 + l];
              aT[2 * (base + l)] += lam * fr;
              aT[2 * (base + l) + 1] += lam * fi;
            }
          }
          if (pol) {
            double qr = FbQ[o], qi = FbQ[o + 1], ur = FbU[o], ui = FbU[o + 1];
            for (int l = (m > 2 ? m : 2); l <= lmax; ++l) {
              double lp = 0.5 * (dp[j * L1 + l] + dm[j * L1 + l]);
              double lmn = 0.5 * (dp[j * L1 + l] - dm[j * L1 + l]);
              /* Ebar += -lp Qb - i lmn Ub ; Bbar += i lmn Qb - lp Ub */
              aE[2 * (base + l)] += -lp * qr + lmn * ui;
              aE[2 * (base + l) + 1] += -lp * qi - lmn * ur;
              aB[2 * (base + l)] += -lmn * qi - lp * ur;
              aB[2 * (base + l) + 1] += lmn * qr - lp * ui;
            }
          }
        }
      }
      if (m == 0) {
        for (int l = 0; l <= lmax; ++l) {
          if (aT) aT[2 * (base + l) + 1] = 0.0;
          if (aE) aE[2 * (base + l) + 1] = 0.0;
          if (aB) aB[2 * (base + l) + 1] = 0.0;
        }
      }
    }
    free(d0); free(dp); free(dm);
  }
}
