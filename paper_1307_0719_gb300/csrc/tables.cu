// Host-side geometry and transform tables (written into caller-provided arrays,
// no allocation). Used by plan creation.
#include <algorithm>
#include <math.h>

#include "common.cuh"

namespace tl {

static const double kPiH = 3.14159265358979323846;

// Polynomials of degree < 16, coefficients in increasing degree.
struct Poly16 {
  double c[16];
  int n;  // number of coefficients
};
static Poly16 poly_deriv(const Poly16 &p) {
  Poly16 d;
  d.n = p.n > 1 ? p.n - 1 : 1;
  for (int i = 0; i < 16; ++i) d.c[i] = 0.0;
  for (int i = 1; i < p.n; ++i) d.c[i - 1] = p.c[i] * (double)i;
  return d;
}
// p * (a + b x^2)
static Poly16 poly_mul_q(const Poly16 &p, double a, double b) {
  Poly16 r;
  r.n = p.n + 2;
  for (int i = 0; i < 16; ++i) r.c[i] = 0.0;
  for (int i = 0; i < p.n; ++i) {
    r.c[i] += a * p.c[i];
    r.c[i + 2] += b * p.c[i];
  }
  return r;
}
static double poly_eval(const Poly16 &p, double x) {
  double r = 0.0;
  for (int i = p.n; i-- > 0;) r = r * x + p.c[i];
  return r;
}

// HEALPix RING rings (Gorski et al. 2005) plus what the Legendre seeds need:
// log2 sin(th/2), log2 cos(th/2) and d^k/dth^k of ln sin(th/2), ln cos(th/2).
// With w = cot(th/2): d/dth ln sin(th/2) = w/2 and dw/dth = -(1+w^2)/2; with
// v = tan(th/2): d/dth ln cos(th/2) = -v/2 and dv/dth = (1+v^2)/2.
void host_ring_tables(int N, const RingHostView &h) {
  const int nr = 4 * N - 1;
  const long long npix = 12LL * N * N, ncap = 2LL * N * (N - 1);
  const int K = TL_MAX_NDER + 1;
  Poly16 ps[TL_MAX_NDER + 2], pc[TL_MAX_NDER + 2];
  for (int i = 0; i < 16; ++i) ps[1].c[i] = pc[1].c[i] = 0.0;
  ps[1].n = pc[1].n = 2;
  ps[1].c[1] = 0.5;
  pc[1].c[1] = -0.5;
  for (int k = 1; k < K; ++k) {
    ps[k + 1] = poly_mul_q(poly_deriv(ps[k]), -0.5, -0.5);
    pc[k + 1] = poly_mul_q(poly_deriv(pc[k]), 0.5, 0.5);
  }
  for (int r = 0; r < nr; ++r) {
    const int i = r + 1;
    const int in = i < 4 * N - i ? i : 4 * N - i;
    double omz_m, omz_p;  // 1 - z and 1 + z, each without cancellation
    double z;
    if (in < N) {
      const double omz = (double)in * in / (3.0 * N * N);
      if (i < 2 * N) { z = 1.0 - omz; omz_m = omz; omz_p = 2.0 - omz; }
      else { z = -(1.0 - omz); omz_m = 2.0 - omz; omz_p = omz; }
      h.nphi[r] = 4 * in;
      h.phi0[r] = kPiH / (4.0 * in);
    } else {
      z = 4.0 / 3.0 - 2.0 * i / (3.0 * N);
      omz_m = 1.0 - z;
      omz_p = 1.0 + z;
      h.nphi[r] = 4 * N;
      h.phi0[r] = ((i - N) % 2 == 0) ? kPiH / (4.0 * N) : 0.0;
    }
    h.inorth[r] = in;
    h.z[r] = z;
    h.dphi[r] = 2.0 * kPiH / (double)h.nphi[r];
    h.omza[r] = omz_m < omz_p ? omz_m : omz_p;
    h.sint[r] = sqrt(omz_m * omz_p);
    h.rsinf[r] = (float)(1.0 / h.sint[r]);
    h.theta[r] = (z >= 0.0) ? 2.0 * asin(sqrt(0.5 * omz_m)) : kPiH - 2.0 * asin(sqrt(0.5 * omz_p));
    {
      float *f = h.ringf + 8 * (size_t)r;
      const float th_hi = (float)h.theta[r];
      f[0] = (float)z;
      f[1] = (float)h.sint[r];
      f[2] = (float)h.omza[r];
      f[3] = th_hi;
      f[4] = (float)(h.theta[r] - (double)th_hi);
      f[5] = f[6] = f[7] = 0.0f;
    }
    h.lsh[r] = 0.5 * log2(0.5 * omz_m);
    h.lch[r] = 0.5 * log2(0.5 * omz_p);
    const double w = sqrt(omz_p / omz_m), v = sqrt(omz_m / omz_p);
    for (int k = 1; k <= K; ++k) {
      h.dls[(size_t)r * K + (k - 1)] = poly_eval(ps[k], w);
      h.dlc[(size_t)r * K + (k - 1)] = poly_eval(pc[k], v);
    }
    if (i < N) h.first[r] = 2LL * i * (i - 1);
    else if (i <= 3 * N) h.first[r] = ncap + (long long)(i - N) * 4 * N;
    else { const long long is = 4LL * N - i; h.first[r] = npix - 2 * is * (is + 1); }
  }
}

// log2 of sqrt((2m+1)/(4 pi)) sqrt(C(2m, m)) = log2 sqrt((2m+1)/4pi) + m + 1/2 sum_k log2((2k-1)/(2k))
void host_lnorm0(int lmax, double *out) {
  double acc = 0.0;
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) acc += log1p(-1.0 / (2.0 * m)) / log(2.0);
    out[m] = 0.5 * log2((2.0 * m + 1.0) / (4.0 * kPiH)) + m + 0.5 * acc;
  }
}

// Bluestein lengths: cap rings use sub-transforms of length i = 1 .. nside-1; each
// non-power-of-two i gets a spectrum of M = pow2 >= 2i - 1 entries followed by its
// chirp of i entries.
long long host_bluestein_layout(int nside, long long *off, int *ml, int *maxm) {
  long long tot = 0;
  int mx = 0;
  for (int i = 0; i <= nside; ++i) {
    off[i] = -1;
    ml[i] = 0;
  }
  for (int i = 1; i < nside; ++i) {
    if ((i & (i - 1)) == 0) continue;
    int M = 1;
    while (M < 2 * i - 1) M <<= 1;
    off[i] = tot;
    ml[i] = M;
    tot += M + i;
    if (M > mx) mx = M;
  }
  *maxm = mx;
  return tot;
}

// Rings of each ring-FFT launch: the equatorial belt, then the caps by Bluestein
// length M (largest first), then the power-of-two caps; each group's rings are
// ordered by decreasing length. No allocation.
int host_fft_groups(int nside, int nrings, const int *nphi, const int *ml, FftGroup *groups, int *order) {
  int ng = 0, n = 0;
  auto key_of = [&](int r) {
    const int ni = nphi[r] / 4;
    return (ni == nside) ? -1 : ((ni & (ni - 1)) == 0 ? 0 : ml[ni]);
  };
  auto add = [&](int key) {
    const int first = n;
    for (int r = 0; r < nrings; ++r)
      if (key_of(r) == key) order[n++] = r;
    if (n == first) return true;
    std::sort(order + first, order + n, [&](int a, int b) { return nphi[a] != nphi[b] ? nphi[a] > nphi[b] : a < b; });
    if (ng == TL_MAX_FFT_GROUPS) return false;
    groups[ng].first = first;
    groups[ng].count = n - first;
    groups[ng].ni_max = nphi[order[first]] / 4;
    groups[ng].ni_min = nphi[order[n - 1]] / 4;
    groups[ng].M = key > 0 ? key : 0;
    ++ng;
    return true;
  };
  if (!add(-1)) return -1;
  for (int M = 1 << 30; M >= 2; M >>= 1)
    if (M <= 4 * nside && !add(M)) return -1;
  if (!add(0)) return -1;
  return n == nrings ? ng : -1;
}

// long enough for every Bluestein length and for a whole belt ring (4 nside), whose
// register FFT takes its first pass's twiddles W_N^j from this table
int host_twiddle_len(int nside, int maxm) {
  int TW = 2;
  while (TW < maxm || TW < 4 * nside) TW <<= 1;
  return TW;
}

// e^{-2 pi i k / TW}, k < TW/2, interleaved (re, im): TW doubles
void host_twiddles(int TW, double *tw) {
  for (int k = 0; k < TW / 2; ++k) {
    const double a = 2.0 * kPiH * (double)k / (double)TW;
    tw[2 * k] = cos(a);
    tw[2 * k + 1] = -sin(a);
  }
}

}  // namespace tl
