// Ring synthesis: from the per-ring Fourier coefficients F^j_m(theta_r) to the
// derivative maps on the ring's equally spaced pixels (Naess & Louis 2013,
// Sec. II.B: the maps d_theta^j d_phi^k s of Eq. 4 at the pixel centres),
//   D(theta_r, phi_p) = Re[ G_0 + 2 sum_{m>0} G_m e^{i m phi_p} ],
//   G_m = (i m)^k F^j_m,  phi_p = phi0_r + 2 pi p / nphi_r.
//
// Per ring, two real output maps (a, b) share one complex inverse DFT of length
// N = nphi = 4i: m is folded modulo N, the spectrum is made Hermitian so that
// the transform of Z = C^a + i C^b is D_a + i D_b, and the DFT is split into four
// length-i transforms of the decimated sequences Z_{4 t1 + t2} followed by one
// radix-4 pass. Length-i transforms use an in-place radix-2 FFT when i is a power
// of two and Bluestein's chirp-z convolution otherwise. All of it runs in shared
// memory; the chirp spectra of Bluestein are tabulated per length at plan time.
#include <math.h>

#include "fft.cuh"
#include "regfft.cuh"

namespace tl {

// One output map: its coefficient plane's first ring (T2 [ring][m], chosen on the
// host, so that the kernel indexes no parameter array at run time), phi-derivative
// order k, 1/sin(theta) weight and output scale (double, and rounded to float).
struct JobDev {
  const void *in;
  void *out;
  double scale;
  float scalef;
  int k, div_sint;
  long long tile;  // output layout: 0 plain, else the tile stride (see d3_pix)
  int il;          // input rows four-ring interleaved (element m at row[4 m])
};

// The ring's coefficient row in a plane and the element stride along m
template <typename T2>
__device__ __forceinline__ const T2 *job_row(const JobDev &J, int r, int mmax, int &fs) {
  fs = J.il ? 4 : 1;
  return J.il ? (const T2 *)J.in + (size_t)(r >> 2) * (size_t)(mmax + 1) * 4 + (r & 3)
              : (const T2 *)J.in + (size_t)r * (mmax + 1);
}
#define TL_MAX_JOBS 96
struct JobList {
  int n;
  JobDev job[TL_MAX_JOBS];
};
// adjoint: one output plane (plane 0..2 = T, Q, U with inputs d_theta^j d_phi^k,
// k < nk, at base + map_index(j, k) npix; plane 3 = phi with one input map at base),
// written at fout (T2 [ring][m], its first ring)
struct AdjJobDev {
  const void *base;
  void *fout;
  int plane, j, nk, pad;
};
#define TL_MAX_ADJ_JOBS 32
struct AdjJobList {
  int n;
  AdjJobDev job[TL_MAX_ADJ_JOBS];
};

// Stride of the four decimated sub-sequences of a ring with nphi = 4 ni: ni for
// power-of-two ni (swizzled layout), else the next value = 4 mod 16.
__host__ __device__ __forceinline__ int ring_sub_stride(int ni) {
  return ((ni & (ni - 1)) == 0) ? ni : ni + ((20 - (ni & 15)) & 15);
}
static int ring_sub_stride_max(const FftGroup &g) {
  int mx = 0;
  for (int ni = g.ni_min; ni <= g.ni_max; ++ni) {
    const int s = ring_sub_stride(ni);
    if (s > mx) mx = s;
  }
  return mx;
}

// The fold sums, over the aliasing class m = t0 + qN (q >= 0, m <= mmax) of a
// ring of N pixels,
//   (-1)^q [shifted rings] * w_m (i m / L)^k F_m,   w_0 = 1, w_m = 2,
// i.e. the class's contribution without its common phase e^{i t0 phi0}.

// x 2^n, exactly
template <typename T> __device__ __forceinline__ T scale2(T x, int n);
template <> __device__ __forceinline__ float scale2<float>(float x, int n) { return scalbnf(x, n); }
template <> __device__ __forceinline__ double scale2<double>(double x, int n) { return scalbn(x, n); }

// (i)^k g
template <typename T2>
__device__ __forceinline__ T2 rot_ik(T2 a, int k) {
  T2 g;
  switch (k & 3) {
    case 0: g = a; break;
    case 1: g.x = -a.y; g.y = a.x; break;
    case 2: g.x = -a.x; g.y = -a.y; break;
    default: g.x = a.y; g.y = -a.x; break;
  }
  return g;
}

// The class sum for the two jobs of a transform in one pass over the class's m: the
// weight, the sign and the power (m/L)^k (built once up to the larger k) are
// shared, and the coefficient row is read once when both jobs read the same
// plane (`same`). The factors 2 and -1 are exact, so the order of the products
// does not change the values.
template <typename T, typename T2>
__device__ __forceinline__ void fold_pair(const T2 *__restrict__ FA, const T2 *__restrict__ FB, bool same,
                                          bool hasb, int t0, int mstep, int mmax, int kA, int kB, T invL,
                                          bool shifted, int qstep_odd, T2 &ga, T2 &gb, int fs) {
  T2 aa, ab;
  aa.x = aa.y = ab.x = ab.y = (T)0;
  const int kmax = (hasb && kB > kA) ? kB : kA;
  int q = 0;
  for (int m = t0; m <= mmax; m += mstep, q += 1) {
    const T2 fa = FA[(size_t)m * fs];
    T2 fb = fa;
    if (hasb && !same) fb = FB[(size_t)m * fs];
    const T mm = (T)m * invL;
    T w = (m > 0) ? (T)2 : (T)1;
    if (shifted && ((q * qstep_odd) & 1)) w = -w;
    T pa = w, pb = w, pw = w;
    for (int r = 1; r <= kmax; ++r) {
      pw *= mm;
      if (r == kA) pa = pw;
      if (r == kB) pb = pw;
    }
    aa.x = fma(fa.x, pa, aa.x);
    aa.y = fma(fa.y, pa, aa.y);
    ab.x = fma(fb.x, pb, ab.x);
    ab.y = fma(fb.y, pb, ab.y);
  }
  ga = rot_ik(aa, kA);
  gb = hasb ? rot_ik(ab, kB) : ab;
}

// Bluestein on the four sub-sequences Y + t2 SY (t2 < 4) of length ni, in place,
//   y_p <- sum_{t < ni} y_t e^{+2 pi i t p / ni}   (what bluestein_batch computes),
// with register passes, for M = 2^LG: the NT threads of the block form NT / (M/16)
// groups; each takes one sub-sequence at a time with its own padded exchange array
// of M elements in W. The chirped input (zero from ni on; ni <= M / 2) goes through a
// forward transform, the product with the length's spectrum (stored in natural
// order, 1/M included, followed by the chirp e^{i pi t^2 / ni}) and an unnormalised
// inverse transform; the chirped outputs p < ni go back to the sub-sequence.
template <int LG, int NT = 512>
__device__ __forceinline__ void reg_bluestein(float2 *Y, int SY, int ni, float2 *W, const float2 *__restrict__ spec,
                                              const float2 *__restrict__ tw, int lgtw) {
  static_assert(LG >= 8 && LG <= 12, "M = 2^8 .. 2^12");
  typedef RegFft<LG, -1> Ff;
  typedef RegFft<LG, +1> Fi;
  constexpr int M = 1 << LG, TGB = M / 16, K = NT / TGB, KK = K < 4 ? K : 4;
  static_assert(K == 1 || K == 2 || K == 4, "one, two or four groups of the block's threads");
  const int tid = threadIdx.x;
  const int grp = tid / TGB, hh = tid - grp * TGB;
  const float2 *__restrict__ chirp = spec + M;
  float2 *xb = W + (size_t)grp * Ff::SMEM;
  for (int round = 0; round < 4 / KK; ++round) {
    float2 *yq = Y + (size_t)(round * KK + grp) * SY;
    float2 x[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int t = hh + TGB * c;
      x[c] = (c < 8 && t < ni) ? cmul(yq[t], __ldg(chirp + t)) : f2(0.0f, 0.0f);
    }
    if constexpr (LG >= 12) {
      // one CTA per SM with the full register file: the table loads of each product
      // are issued before the transform that precedes it, so they overlap its passes
      float2 bq[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) bq[c] = __ldg(spec + hh + TGB * c);
      Ff::run(x, xb, hh, tw, lgtw);
#pragma unroll
      for (int c = 0; c < 16; ++c) x[c] = cmul(x[c], bq[c]);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int pp = hh + TGB * c;
        bq[c] = pp < ni ? __ldg(chirp + pp) : f2(0.0f, 0.0f);
      }
      Fi::run(x, xb, hh, tw, lgtw);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int pp = hh + TGB * c;
        if (pp < ni) yq[pp] = cmul(x[c], bq[c]);
      }
    } else {
      Ff::run(x, xb, hh, tw, lgtw);
#pragma unroll
      for (int c = 0; c < 16; ++c) x[c] = cmul(x[c], __ldg(spec + hh + TGB * c));
      Fi::run(x, xb, hh, tw, lgtw);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int pp = hh + TGB * c;
        if (pp < ni) yq[pp] = cmul(x[c], __ldg(chirp + pp));
      }
    }
  }
  __syncthreads();
}

// BLUE: the launch's rings have non-power-of-two sub-transforms (Bluestein); else
// power-of-two ones. REG: Bluestein by register passes (reg_bluestein; see ring_threads). A launch covers one ring group, so each instance carries one
// sub-transform path (and its own register allocation). LG > 0: the group's
// transform length is known at compile time, 2^LG (power-of-two rings: the
// sub-transform length ni; Bluestein: the convolution length M), so the FFT's index
// and address arithmetic folds into constants; LG = 0 takes it from the ring.
// threads of a ring-FFT CTA: 256 for the register Bluestein (M = 2^12: one
// sub-transform at a time, 100 KB of shared memory, two CTAs per SM at 128 registers;
// M = 2^11: two at a time, 68 KB, three CTAs per SM), so that the CTAs' phases
// (fold from HBM, transforms, output pass) interleave; else 512
template <bool REG, int LG> constexpr int ring_threads() { return (REG && LG >= 11) ? 256 : 512; }
// CTAs per SM the register allocation is held to: M = 2^11 fits three (68 KB of shared
// memory each), M = 2^12 two
template <typename T, bool REG, int LG> constexpr int ring_min_ctas() {
  return sizeof(T) != 4 ? 1 : (REG && LG == 11) ? 3 : 2;
}

template <typename T, bool BLUE, int LG = 0, bool REG = false>
__global__ void __launch_bounds__(ring_threads<REG, LG>(), ring_min_ctas<T, REG, LG>()) ringfft_kernel(RingTable rt, int nside, int mmax, JobList jobs,
                                                      BluesteinTable bt,
                                                      const typename RealTraits<T>::T2 *__restrict__ tw, int TW,
                                                      int bbatch, T invL, const int *__restrict__ rings,
                                                      const typename RealTraits<T>::T2 *__restrict__ phase) {
  typedef typename RealTraits<T>::T2 T2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = rings[blockIdx.x];
  const int pair = blockIdx.y;
  const int ja = 2 * pair, jb = 2 * pair + 1;
  const bool hasb = jb < jobs.n;
  constexpr bool LGP = LG > 0 && !BLUE;  // power-of-two rings of one known length
  const int N = LGP ? (4 << LG) : rt.nphi[r];
  const int ni = N >> 2;
  const int half = N >> 1;
  const long long first = rt.first[r];
  const int nth = blockDim.x, tid = threadIdx.x;
  // Y: the four decimated sub-sequences Z_{4 t1 + t2}, SY apart. Power-of-two ni: the
  // swizzled layout, stored in bit-reversed order (the input order of the in-place
  // FFT); other ni: plain, with SY = 4 mod 16 so that the four arrays fall on
  // different banks.
  const bool pw2 = !BLUE;  // the group is of one kind: (ni & (ni - 1)) == 0 iff !BLUE
  const int lgni = LGP ? LG : 31 - __clz(ni);
  const int SY = LGP ? (1 << LG) : ring_sub_stride(ni);
  T2 *Y = (T2 *)smem_raw;
  T2 *W = Y + 4 * SY;  // work area
  const bool yswz = pw2 && ni >= 16;  // the XOR layout needs whole 16-element blocks
  auto yaddr = [&](int b, int i) { return yswz ? faddr(b, i, lgni, SY) : b * SY + i; };
  auto ydst = [&](int t) { return yaddr(t & 3, pw2 ? brev_bits(t >> 2, lgni) : (t >> 2)); };
  // half-pixel-shifted rings have phi0 = pi / (4 ni) = pi / N: e^{i m phi0} = e^{i t phi0} (-1)^q
  // for m = t + q N
  const bool shifted = __double_as_longlong(rt.phi0[r]) != 0;  // phi0 >= 0: an integer test

  const JobDev JA = jobs.job[ja];
  const JobDev JB = hasb ? jobs.job[jb] : jobs.job[ja];
  int fs;
  const T2 *FA = job_row<T2>(JA, r, mmax, fs);
  const T2 *FB = job_row<T2>(JB, r, mmax, fs);
  const bool same = JA.in == JB.in;  // both maps from one coefficient plane (different k)
  // both packed maps are transformed in the normalised units of the Legendre stage
  // (similar magnitudes, so the shared transform's rounding does not leak from a
  // large map into a small one); each job's scale is applied on output
  // single precision takes its per-ring and per-job factors from float tables: a
  // double operation per thread would queue on the FP64 pipe
  constexpr bool F32 = sizeof(T) == 4;
  const T inv_s = F32 ? (T)rt.rsinf[r] : (T)(1.0 / rt.sint[r]);
  T wa = JA.div_sint ? inv_s : (T)1;
  T wb = hasb ? (JB.div_sint ? inv_s : (T)1) : (T)0;
  T sa = F32 ? (T)JA.scalef : (T)JA.scale, sb = F32 ? (T)JB.scalef : (T)JB.scale;
  // Balance of the two packed maps. A normalised phi-derivative map scales like
  // (m/L)^k, and near the poles only m up to about L sin(theta) contribute, so there
  // map k is ~ (L sin th)^-k times map 0 and a shared transform's rounding of the
  // larger map would swamp the smaller one. Each job is carried times 2^(e k') in the
  // transform (k' = k, less one for a map divided by sin theta, which that division
  // already balances), 2^e ~ L / (1 + L sin th), and scaled back on output: powers
  // of two, so the values are unchanged.
  {
    const float Lf = (float)((T)1 / invL), sf = rt.ringf[8 * (size_t)r + 1];
    const int e = max(0, __float2int_rn(log2f(Lf / (1.0f + Lf * sf))));
    const int ea = e * max(0, JA.k - JA.div_sint), eb = e * max(0, JB.k - JB.div_sint);
    wa = scale2<T>(wa, ea);
    wb = scale2<T>(wb, eb);
    sa = scale2<T>(sa, -ea);
    sb = scale2<T>(sb, -eb);
  }
  const T invN = (T)1 / (T)N;
  // e^{i pi t / N}, t = 0 .. N/2, of this ring's length (plan-time table, see phase_table_kernel)
  const T2 *__restrict__ eph = phase + ((size_t)ni * ni - 1);

  // ---- fold m modulo N into the Hermitian spectrum; thread handles classes t and N - t
  // (t = 0 .. N/2): C_t = (B_t + conj(B_{-t}))/2, C_{-t} = conj(C_t), Z = C^a + i C^b.
  // Z_t is stored at sub-sequence t % 4, element t / 4 (see ydst).
  const int ncls = half + 1;
  const int C = (ncls >= nth) ? 1 : nth / ncls;  // threads sharing one class pair
  // class pair (t, N - t) from its sums Ba, Bam (map a) and Bb, Bbm (map b) over
  // chunk c of the aliasing terms: class phases, Hermitian combination, store
  auto finish = [&](int tt, int c, T2 Ba, T2 Bam, T2 Bb, T2 Bbm) {
    const int tm = tt ? N - tt : 0;
    // chunk c starts at q = c: its first sign is (-1)^c on shifted rings
    if (shifted && (c & 1)) {
      Ba.x = -Ba.x; Ba.y = -Ba.y; Bam.x = -Bam.x; Bam.y = -Bam.y;
      Bb.x = -Bb.x; Bb.y = -Bb.y; Bbm.x = -Bbm.x; Bbm.y = -Bbm.y;
    }
    if (shifted) {
      // class phases e^{i t phi0} and e^{i (N-t) phi0} = -conj(e^{i t phi0}) (t > 0)
      const T2 e = eph[tt];
      T2 em;
      if (tt == 0) em = e;
      else {
        em.x = -e.x;
        em.y = e.y;
      }
      Ba = cmul(Ba, e);
      Bb = cmul(Bb, e);
      Bam = cmul(Bam, em);
      Bbm = cmul(Bbm, em);
    }
    T2 ca, cb;  // C^a_t, C^b_t (weights of the maps included)
    ca.x = (T)0.5 * wa * (Ba.x + Bam.x);
    ca.y = (T)0.5 * wa * (Ba.y - Bam.y);
    cb.x = (T)0.5 * wb * (Bb.x + Bbm.x);
    cb.y = (T)0.5 * wb * (Bb.y - Bbm.y);
    if (C == 1) {
      T2 z, zm;
      z.x = ca.x - cb.y;
      z.y = ca.y + cb.x;
      zm.x = ca.x + cb.y;  // conj(C^a) + i conj(C^b)
      zm.y = -ca.y + cb.x;
      Y[ydst(tt)] = z;
      if (tt != 0 && tt != half) Y[ydst(tm)] = zm;
    } else {
      W[2 * (c * ncls + tt)] = ca;
      W[2 * (c * ncls + tt) + 1] = cb;
    }
  };
  if (C == 1 && N > mmax) {
    // no aliasing: class t has at most the term m = t, class N - t the term
    // m = N - t (q = 0). A chunk of classes' coefficients is loaded first, then
    // weighed (as fold_pair does, with the same roundings) and stored.
    constexpr int U = 4;
    const int kmax = (hasb && JB.k > JA.k) ? JB.k : JA.k;
    T2 zero;
    zero.x = zero.y = (T)0;
    auto weigh = [&](T2 fa, T2 fb, int m, T2 &ga, T2 &gb) {
      const T mm = (T)m * invL;
      const T w = (m > 0) ? (T)2 : (T)1;
      T pa = w, pb = w, pw = w;
      for (int r = 1; r <= kmax; ++r) {
        pw *= mm;
        if (r == JA.k) pa = pw;
        if (r == JB.k) pb = pw;
      }
      T2 x, y;
      x.x = fa.x * pa;
      x.y = fa.y * pa;
      y.x = fb.x * pb;
      y.y = fb.y * pb;
      ga = rot_ik(x, JA.k);
      gb = hasb ? rot_ik(y, JB.k) : zero;
    };
    for (int t0 = tid; t0 < ncls; t0 += U * nth) {
      T2 fa[U], fb[U], fam[U], fbm[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int tt = t0 + u * nth;
        const int tm = tt ? N - tt : 0;
        const bool lo = tt < ncls && tt <= mmax, hi = tt < ncls && tm <= mmax;
        fa[u] = lo ? FA[(size_t)tt * fs] : zero;
        fam[u] = hi ? FA[(size_t)tm * fs] : zero;
        fb[u] = (hasb && !same && lo) ? FB[(size_t)tt * fs] : fa[u];
        fbm[u] = (hasb && !same && hi) ? FB[(size_t)tm * fs] : fam[u];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int tt = t0 + u * nth;
        if (tt >= ncls) break;
        T2 Ba, Bb, Bam, Bbm;
        weigh(fa[u], fb[u], tt, Ba, Bb);
        weigh(fam[u], fbm[u], tt ? N - tt : 0, Bam, Bbm);
        finish(tt, 0, Ba, Bam, Bb, Bbm);
      }
    }
  } else {
    const int c = tid / ncls, t = tid - (tid / ncls) * ncls;
    for (int tt = (C == 1 ? tid : t); tt < ncls && c < C; tt += (C == 1 ? nth : ncls)) {
      const int tm = tt ? N - tt : 0;
      const int m0 = tt + c * N, m1 = tm + c * N, step = C * N;
      T2 Ba, Bb, Bam, Bbm;
      fold_pair<T, T2>(FA, FB, same, hasb, m0, step, mmax, JA.k, JB.k, invL, shifted, C, Ba, Bb, fs);
      fold_pair<T, T2>(FA, FB, same, hasb, m1, step, mmax, JA.k, JB.k, invL, shifted, C, Bam, Bbm, fs);
      if (!hasb) Bb.x = Bb.y = Bbm.x = Bbm.y = (T)0;
      finish(tt, c, Ba, Bam, Bb, Bbm);
    }
  }
  if (C > 1) {
    __syncthreads();
    for (int tt = tid; tt < ncls; tt += nth) {
      T2 ca = {0, 0}, cb = {0, 0};
      for (int c = 0; c < C; ++c) {
        ca = cadd(ca, W[2 * (c * ncls + tt)]);
        cb = cadd(cb, W[2 * (c * ncls + tt) + 1]);
      }
      const int tm = tt ? N - tt : 0;
      T2 z, zm;
      z.x = ca.x - cb.y;
      z.y = ca.y + cb.x;
      zm.x = ca.x + cb.y;
      zm.y = -ca.y + cb.x;
      Y[ydst(tt)] = z;
      if (tt != 0 && tt != half) Y[ydst(tm)] = zm;
    }
  }
  __syncthreads();

  // ---- four length-ni inverse DFTs
  if (!BLUE) {
    if (yswz)
      fft_core<true, T, T2, LGP ? LG : 0>(Y, ni, 4, SY, +1, tw, TW);
    else
      fft_core<false, T, T2, LGP ? LG : 0>(Y, ni, 4, SY, +1, tw, TW);
  } else if constexpr (REG) {
    reg_bluestein<LG, ring_threads<REG, LG>()>((float2 *)Y, SY, ni, (float2 *)W,
                                               (const float2 *)bt.spec + bt.offset[ni], (const float2 *)tw,
                                               31 - __clz(TW));
  } else {
    const long long off = bt.offset[ni];
    const int M = LG ? (1 << LG) : bt.mlen[ni];
    const T2 *bh = (const T2 *)bt.spec + off;
    const T2 *ch = bh + M;  // the length's chirp follows its spectrum
    const int SW = M;
    if (bbatch >= 4) {
      bluestein_batch<T, T2, LG>(Y, ni, SY, M, 4, W, SW, bh, ch, tw, TW);
    } else {
      for (int t2 = 0; t2 < 4; ++t2)
        bluestein_batch<T, T2, LG>(Y + t2 * SY, ni, SY, M, 1, W, SW, bh, ch, tw, TW);
    }
  }

  // ---- radix-4 pass: X_{p1 + ni p2} = sum_t2 i^{t2 p2} e^{2 pi i t2 p1 / N} Y_t2(p1)
  T *outA = (T *)JA.out;
  T *outB = hasb ? (T *)JB.out : nullptr;
  // output index of ring pixel p (plain, or the pixel-tiled layout of the plan's maps)
  auto oidx = [&](long long tile, int p) -> long long {
    const long long g = first + p;
    return tile ? d3_pix(g, tile) : g;
  };
  for (int p1 = tid; p1 < ni; p1 += nth) {
    const T2 w1 = eph[2 * p1];  // e^{2 pi i p1 / N}
    const T2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
    T2 y[4];
    y[0] = Y[yaddr(0, p1)];
    y[1] = cmul(Y[yaddr(1, p1)], w1);
    y[2] = cmul(Y[yaddr(2, p1)], w2);
    y[3] = cmul(Y[yaddr(3, p1)], w3);
    const T2 a0 = cadd(y[0], y[2]), a1 = csub(y[0], y[2]);
    const T2 b0 = cadd(y[1], y[3]), b1 = csub(y[1], y[3]);
    T2 ib1;  // i * b1
    ib1.x = -b1.y;
    ib1.y = b1.x;
    const T2 X0 = cadd(a0, b0), X2 = csub(a0, b0);
    const T2 X1 = cadd(a1, ib1), X3 = csub(a1, ib1);
    outA[oidx(JA.tile, p1)] = sa * X0.x;
    outA[oidx(JA.tile, p1 + ni)] = sa * X1.x;
    outA[oidx(JA.tile, p1 + 2 * ni)] = sa * X2.x;
    outA[oidx(JA.tile, p1 + 3 * ni)] = sa * X3.x;
    if (hasb) {
      outB[oidx(JB.tile, p1)] = sb * X0.y;
      outB[oidx(JB.tile, p1 + ni)] = sb * X1.y;
      outB[oidx(JB.tile, p1 + 2 * ni)] = sb * X2.y;
      outB[oidx(JB.tile, p1 + 3 * ni)] = sb * X3.y;
    }
  }
}

// ---------------------------------------------------------------------------
// Rings of N = 2^LG pixels without aliasing (N > mmax), single precision: one CTA of
// N / 16 threads per (ring, pair of output maps). The fold is formed straight in the
// registers of the first FFT pass (thread h, slot c: Z_t with t = h + (N/16) c), the
// register passes of RegFft run the inverse DFT, and each thread stores its sixteen
// outputs. Per output class t, with class t holding m1 = t and class N - t holding
// m2 = N - t (m2 = 0 for t = 0), each present when m <= mmax:
//   Z_t = e_t [ u_a p_a(m1) F^a_m1 + u_b p_b(m1) F^b_m1
//               + sigma conj(u_a p_a(m2) F^a_m2 - u_b p_b(m2) F^b_m2) ],
// u_a = w_a i^k_a / 2, u_b = i w_b i^k_b / 2 (w: the job's 1/sin(theta) weight and
// balance), p(m) = w_m (m / L)^k, e_t = e^{i pi t / N} and sigma = -1 on
// half-pixel-shifted rings (t > 0), e_t = sigma = 1 otherwise: the class sums and
// the Hermitian split of the shared-memory kernel above, written per class.
template <int LG>
__global__ void __launch_bounds__(1 << (LG - 4), 1024 >> (LG - 4))
    ringfft_reg_kernel(RingTable rt, int mmax, JobList jobs, const float2 *__restrict__ tw, int lgtw, float invL,
                       const int *__restrict__ rings, const float2 *__restrict__ phase) {
  typedef RegFft<LG, +1> F;
  constexpr int N = F::N, TG = F::TG, HALF = N / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *sm = (float2 *)smem_raw;
  const int r = rings[blockIdx.x];
  const int pair = blockIdx.y, ja = 2 * pair, jb = 2 * pair + 1;
  const bool hasb = jb < jobs.n;
  const int h = threadIdx.x;
  const long long first = rt.first[r];
  const bool shifted = __double_as_longlong(rt.phi0[r]) != 0;
  const JobDev JA = jobs.job[ja];
  const JobDev JB = hasb ? jobs.job[jb] : jobs.job[ja];
  int fs;
  const float2 *FA = job_row<float2>(JA, r, mmax, fs);
  const float2 *FB = job_row<float2>(JB, r, mmax, fs);
  const bool same = JA.in == JB.in;
  const float inv_s = rt.rsinf[r];
  float wa = JA.div_sint ? inv_s : 1.0f;
  float wb = hasb ? (JB.div_sint ? inv_s : 1.0f) : 0.0f;
  float sa = JA.scalef, sb = JB.scalef;
  {  // magnitude balance of the packed maps, as in ringfft_kernel
    const float Lf = 1.0f / invL, sf = rt.ringf[8 * (size_t)r + 1];
    const int e = max(0, __float2int_rn(log2f(Lf / (1.0f + Lf * sf))));
    const int ea = e * max(0, JA.k - JA.div_sint), eb = e * max(0, JB.k - JB.div_sint);
    wa = scalbnf(wa, ea);
    wb = scalbnf(wb, eb);
    sa = scalbnf(sa, -ea);
    sb = scalbnf(sb, -eb);
  }
  const int kA = JA.k, kB = hasb ? JB.k : 0;
  const int klo = min(kA, kB), khi = max(kA, kB);
  const float2 ua = rot_ik(f2(0.5f * wa, 0.0f), kA);
  const float2 ub = rot_ik(f2(0.5f * wb, 0.0f), kB + 1);
  const float2 *__restrict__ eph = phase + ((size_t)(N / 4) * (N / 4) - 1);  // e^{i pi t / N}, t <= N/2

  // w_m (m / L)^k for the two jobs: binary powers (k <= 7), no loops
  auto powers = [&](int m, float &pa, float &pb) {
    const float m1 = (float)m * invL, m2 = m1 * m1, m4 = m2 * m2;
    const float w = (m > 0) ? 2.0f : 1.0f;
    pa = w;
    pb = w;
    if (kA & 1) pa *= m1;
    if (kA & 2) pa *= m2;
    if (kA & 4) pa *= m4;
    if (kB & 1) pb *= m1;
    if (kB & 2) pb *= m2;
    if (kB & 4) pb *= m4;
  };
  // u_a p_a(m) F^a_m + s u_b p_b(m) F^b_m (s = +1: the class's own term; -1 inside
  // the conjugate of the partner class's term)
  auto comb = [&](int m, float2 fa, float2 fb, float s) -> float2 {
    float pa, pb;
    powers(m, pa, pb);
    const float2 ta = cmul(ua, f2(pa * fa.x, pa * fa.y));
    const float2 tb = cmul(ub, f2(pb * fb.x, pb * fb.y));
    return f2(fmaf(s, tb.x, ta.x), fmaf(s, tb.y, ta.y));
  };
  const float sg = shifted ? -1.0f : 1.0f;  // sigma of the classes t > 0
  const float2 zero = f2(0.0f, 0.0f);
  float2 x[16];
  if (mmax <= HALF && same) {
    // Slot c < 8 (t < N/2) holds class t's own term only, slot c >= 8 (t >= N/2) the
    // conjugate of class N - t's only: one coefficient per slot (both maps read one
    // plane), all sixteen loads in flight before the arithmetic, which then runs in
    // place. Classes 0 and N/2 get their other term below.
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int t = h + TG * c;
      const int m = c < 8 ? t : N - t;
      x[c] = m <= mmax ? __ldg(FA + (size_t)m * fs) : zero;
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int t = h + TG * c;
      if (c < 8) {
        x[c] = comb(t, x[c], x[c], 1.0f);
      } else {
        const float2 d = comb(N - t, x[c], x[c], -1.0f);
        x[c] = f2(sg * d.x, -sg * d.y);
      }
    }
    if (h == 0) {
      const float2 f0 = __ldg(FA);
      const float2 d0 = comb(0, f0, f0, -1.0f);
      x[0] = f2(x[0].x + d0.x, x[0].y - d0.y);
      if (HALF <= mmax) {
        const float2 fa = __ldg(FA + (size_t)HALF * fs);
        x[8] = cadd(x[8], comb(HALF, fa, fa, 1.0f));
      }
    }
  } else if (mmax <= HALF) {
    // as above with two coefficient rows: two batches of eight slots
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float2 va[8], vb[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = h + TG * (8 * half + u);
        const int m = half ? N - t : t;
        const bool ok = m <= mmax;
        va[u] = ok ? __ldg(FA + (size_t)m * fs) : zero;
        vb[u] = (ok && !same) ? __ldg(FB + (size_t)m * fs) : va[u];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = h + TG * (8 * half + u);
        if (half == 0) {
          x[u] = comb(t, va[u], vb[u], 1.0f);
        } else {
          const float2 d = comb(N - t, va[u], vb[u], -1.0f);
          x[8 + u] = f2(sg * d.x, -sg * d.y);
        }
      }
    }
    if (h == 0) {
      // t = 0: the partner class is class 0 itself (sigma = +1)
      const float2 d0 = comb(0, __ldg(FA), same ? __ldg(FA) : __ldg(FB), -1.0f);
      x[0] = f2(x[0].x + d0.x, x[0].y - d0.y);
      // t = N/2: class N/2's own term m = N/2
      if (HALF <= mmax) {
        const float2 fa = __ldg(FA + (size_t)HALF * fs);
        x[8] = cadd(x[8], comb(HALF, fa, same ? fa : __ldg(FB + (size_t)HALF * fs), 1.0f));
      }
    }
  } else {
    // band limit above N/2: both terms wherever m <= mmax
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int t = h + TG * c;
      const int m2 = t ? N - t : 0;
      float2 z = zero;
      if (t <= mmax) {
        const float2 fa = __ldg(FA + (size_t)t * fs);
        z = comb(t, fa, same ? fa : __ldg(FB + (size_t)t * fs), 1.0f);
      }
      if (m2 <= mmax) {
        const float2 fa = __ldg(FA + (size_t)m2 * fs);
        const float2 d = comb(m2, fa, same ? fa : __ldg(FB + (size_t)m2 * fs), -1.0f);
        const float s2 = t ? sg : 1.0f;
        z.x = fmaf(s2, d.x, z.x);
        z.y = fmaf(-s2, d.y, z.y);
      }
      x[c] = z;
    }
  }
  if (shifted) {
    // e_t = e^{i pi t / N} = e_h e^{i pi c / 16} (t = h + (N/16) c)
    // cos, sin of pi c / 16
    constexpr float kc[16] = {1.00000000000000000000f, 0.98078528040323043058f, 0.92387953251128673848f, 0.83146961230254523567f, 0.70710678118654757274f, 0.55557023301960228867f, 0.38268343236508983729f, 0.19509032201612833135f, 0.00000000000000006123f, -0.19509032201612819257f, -0.38268343236508972627f, -0.55557023301960195560f, -0.70710678118654746172f, -0.83146961230254534669f, -0.92387953251128673848f, -0.98078528040323043058f};
    constexpr float ks[16] = {0.00000000000000000000f, 0.19509032201612824808f, 0.38268343236508978178f, 0.55557023301960217765f, 0.70710678118654746172f, 0.83146961230254523567f, 0.92387953251128673848f, 0.98078528040323043058f, 1.00000000000000000000f, 0.98078528040323043058f, 0.92387953251128673848f, 0.83146961230254545772f, 0.70710678118654757274f, 0.55557023301960217765f, 0.38268343236508989280f, 0.19509032201612860891f};
    const float2 eh = __ldg(eph + h);
#pragma unroll
    for (int c = 0; c < 16; ++c) x[c] = cmul(x[c], cmul(eh, f2(kc[c], ks[c])));
  }
  F::run(x, sm, h, tw, lgtw);
  float *outA = (float *)JA.out;
  float *outB = hasb ? (float *)JB.out : nullptr;
  const long long tile = JA.tile;  // one layout for every job of a launch
  // The ring starts a tile (the host launches this kernel only for such rings), so
  // pixel h + TG c sits in tile first / 256 + (h + TG c) / 256 at (h + TG c) mod 256.
  // For TG >= 256 that is tile (h / 256) + (TG / 256) c at h mod 256; for TG < 256,
  // h + TG (c mod 256/TG) < 256, so it is tile (TG c) / 256 at h + TG (c mod 256/TG).
  // Plain maps: first + h + TG c.
  constexpr int PER = TG >= kD3Tile ? 1 : kD3Tile / TG;
  const long long base =
      tile ? ((first >> kD3TileLg) + (TG >= kD3Tile ? (h >> kD3TileLg) : 0)) * tile +
                 (TG >= kD3Tile ? (h & (kD3Tile - 1)) : h)
           : first + h;
  float *oa = outA + base;
  float *ob = hasb ? outB + base : nullptr;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const long long off =
        tile ? (long long)((TG * c) >> kD3TileLg) * tile + (TG >= kD3Tile ? 0 : TG * (c % PER)) : (long long)TG * c;
    oa[off] = sa * x[c].x;
    if (hasb) ob[off] = sb * x[c].y;
  }
}

// ---------------------------------------------------------------------------
// Adjoint of the ring synthesis. For an output plane (field, j) fed by the real
// maps g_k (k = derivative order in phi, scale c_k, optional 1/sin(theta)), the
// gradient with respect to the plane's coefficients is
//     Fbar^j_m = w_m e^{-i m phi0} sum_k c_k (-i m / L)^k X^k_{m mod N},
//     X^k_t = sum_p g_k(p) e^{-2 pi i t p / N},
// (the forward map is Re[c w_m (i m/L)^k F_m e^{i m phi_p}], whose gradient in
// the convention dL/dRe + i dL/dIm is the complex conjugate of the factor).
// Two maps share one forward DFT: with Z = g_a + i g_b, X^a_t = (Z_t + conj Z_{N-t})/2,
// X^b_t = (Z_t - conj Z_{N-t})/(2i); the DFT is conj(IDFT(conj Z)), computed by
// the forward kernel's decimated sub-transforms and an in-place radix-4 pass.

template <typename T>
__global__ void __launch_bounds__(512, (sizeof(T) == 4 ? 2 : 1)) ringfft_adj_kernel(RingTable rt, int mmax, long long npix, int nmaps,
                                                          AdjJobList jobs,
                                                          BluesteinTable bt,
                                                          const typename RealTraits<T>::T2 *__restrict__ tw, int TW,
                                                          int bbatch, double L_d, const int *__restrict__ rings,
                                                          const typename RealTraits<T>::T2 *__restrict__ phase,
                                                          int reg_lg) {
  typedef typename RealTraits<T>::T2 T2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = rings[blockIdx.x];
  const AdjJobDev J = jobs.job[blockIdx.y];
  const int N = rt.nphi[r];
  const int ni = N >> 2;
  const long long first = rt.first[r];
  const int nth = blockDim.x, tid = threadIdx.x;
  const bool pw2 = (ni & (ni - 1)) == 0;
  const int lgni = 31 - __clz(ni);
  const int SY = ring_sub_stride(ni);
  T2 *Y = (T2 *)smem_raw;  // the four sub-sequences (layout as in the forward kernel)
  T2 *W = Y + 4 * SY;
  const bool yswz = pw2 && ni >= 16;  // the XOR layout needs whole 16-element blocks
  auto yaddr = [&](int b, int i) { return yswz ? faddr(b, i, lgni, SY) : b * SY + i; };
  auto ydst = [&](int t) { return yaddr(t & 3, pw2 ? brev_bits(t >> 2, lgni) : (t >> 2)); };
  const T2 *__restrict__ eph = phase + ((size_t)ni * ni - 1);  // e^{i pi t / N}, t <= N/2
  const bool shifted = __double_as_longlong(rt.phi0[r]) != 0;  // phi0 = pi / N
  const T invL = (T)(1.0 / L_d);
  const T inv_s = (T)1 / (T)rt.sint[r];
  T2 *F = (T2 *)J.fout + (size_t)r * (mmax + 1);
  // inputs: field planes take k = 0 .. nk-1 with c_k = 1/(j! k!); the deflection's
  // planes one map each (j = 1: k = 0; j = 0: k = 1 over sin(theta)), c = L
  const bool defl = J.plane == 3;
  const int nin = defl ? 1 : J.nk;
  T jfact = (T)1;
  for (int i = 2; i <= J.j; ++i) jfact *= (T)i;

  for (int i0 = 0; i0 < nin; i0 += 2) {
    const bool hasb = i0 + 1 < nin;
    int ka, kb;
    const T *ga, *gb;
    T ca, cb;
    if (defl) {
      ka = kb = (J.j == 0) ? 1 : 0;
      ga = gb = (const T *)J.base;
      ca = (T)L_d * ((J.j == 0) ? inv_s : (T)1);
      cb = (T)0;
    } else {
      ka = i0;
      kb = hasb ? i0 + 1 : i0;
      const int na = (J.j + ka) * (J.j + ka + 1) / 2 + J.j, nb = (J.j + kb) * (J.j + kb + 1) / 2 + J.j;
      ga = (const T *)J.base + (size_t)na * npix;
      gb = (const T *)J.base + (size_t)nb * npix;
      T kfa = (T)1, kfb = (T)1;
      for (int i = 2; i <= ka; ++i) kfa *= (T)i;
      for (int i = 2; i <= kb; ++i) kfb *= (T)i;
      ca = (T)1 / (jfact * kfa);
      cb = hasb ? (T)1 / (jfact * kfb) : (T)0;
    }
    // balance of the packed pair (the transpose of the forward kernel's): near the
    // poles the gradient of map k scales like (L sin th)^k; map k is carried times
    // 2^-(e k) in the transform and its factor c_k times 2^(e k) (exact)
    int ea = 0, eb = 0;
    if (!defl) {
      const float Lf = (float)L_d, sf = rt.ringf[8 * (size_t)r + 1];
      const int e = max(0, __float2int_rn(log2f(Lf / (1.0f + Lf * sf))));
      ea = e * ka;
      eb = e * kb;
      ca = scale2<T>(ca, ea);
      cb = scale2<T>(cb, eb);
    }
    // conj(Z) in decimated order
    for (int p = tid; p < N; p += nth) {
      T2 z;
      z.x = scale2<T>(ga[first + p], -ea);
      z.y = hasb ? -scale2<T>(gb[first + p], -eb) : (T)0;
      Y[ydst(p)] = z;
    }
    __syncthreads();
    if (pw2) {
      if (yswz)
        fft_core<true, T, T2>(Y, ni, 4, SY, +1, tw, TW);
      else
        fft_core<false, T, T2>(Y, ni, 4, SY, +1, tw, TW);
    } else {
      const long long off = bt.offset[ni];
      const int M = bt.mlen[ni];
      const T2 *bh = (const T2 *)bt.spec + off;
      const T2 *ch = bh + M;
      const int SW = M;
      const int lgM = 31 - __clz(M);
      bool done = false;
      if constexpr (sizeof(T) == 4) {
        // the lengths whose spectra are stored for the register passes
        if (reg_lg > 0 && lgM >= reg_lg && lgM <= 12) {
          if (lgM == 12)
            reg_bluestein<12>((float2 *)Y, SY, ni, (float2 *)W, (const float2 *)bh, (const float2 *)tw, 31 - __clz(TW));
          else
            reg_bluestein<11>((float2 *)Y, SY, ni, (float2 *)W, (const float2 *)bh, (const float2 *)tw, 31 - __clz(TW));
          done = true;
        }
      }
      if (done) {
      } else if (bbatch >= 4) {
        bluestein_batch<T, T2>(Y, ni, SY, M, 4, W, SW, bh, ch, tw, TW);
      } else {
        for (int t2 = 0; t2 < 4; ++t2) bluestein_batch<T, T2>(Y + t2 * SY, ni, SY, M, 1, W, SW, bh, ch, tw, TW);
      }
    }
    // radix-4 pass in place (slots p1 + ni t2 are read and written by one thread), then conj
    for (int p1 = tid; p1 < ni; p1 += nth) {
      const T2 w1 = eph[2 * p1];  // e^{2 pi i p1 / N}
      const T2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
      T2 y[4];
      y[0] = Y[yaddr(0, p1)];
      y[1] = cmul(Y[yaddr(1, p1)], w1);
      y[2] = cmul(Y[yaddr(2, p1)], w2);
      y[3] = cmul(Y[yaddr(3, p1)], w3);
      const T2 a0 = cadd(y[0], y[2]), a1 = csub(y[0], y[2]);
      const T2 b0 = cadd(y[1], y[3]), b1 = csub(y[1], y[3]);
      T2 ib1;
      ib1.x = -b1.y;
      ib1.y = b1.x;
      T2 X0 = cadd(a0, b0), X2 = csub(a0, b0);
      T2 X1 = cadd(a1, ib1), X3 = csub(a1, ib1);
      X0.y = -X0.y;
      X1.y = -X1.y;
      X2.y = -X2.y;
      X3.y = -X3.y;
      Y[yaddr(0, p1)] = X0;
      Y[yaddr(1, p1)] = X1;
      Y[yaddr(2, p1)] = X2;
      Y[yaddr(3, p1)] = X3;
    }
    __syncthreads();
    // split the packed spectra and accumulate the plane's row
    for (int m = tid; m <= mmax; m += nth) {
      const int t = m % N;
      const int tm = (N - t) % N;
      const T2 zt = Y[yaddr(t / ni, t % ni)], zm = Y[yaddr(tm / ni, tm % ni)];
      // X^a = (Z_t + conj Z_{N-t})/2, X^b = (Z_t - conj Z_{N-t})/(2i)
      T2 xa, xb;
      xa.x = (T)0.5 * (zt.x + zm.x);
      xa.y = (T)0.5 * (zt.y - zm.y);
      xb.x = (T)0.5 * (zt.y + zm.y);
      xb.y = (T)-0.5 * (zt.x - zm.x);
      // c (m/L)^k (-i)^k X
      const T mm = (T)m * invL;
      T pa = ca, pb = cb;
      for (int i = 0; i < ka; ++i) pa *= mm;
      for (int i = 0; i < kb; ++i) pb *= mm;
      T2 va, vb;
      va.x = pa * xa.x;
      va.y = pa * xa.y;
      vb.x = pb * xb.x;
      vb.y = pb * xb.y;
      T2 v;
      {
        T2 ra, rb;  // multiply by (-i)^k
        switch (ka & 3) {
          case 0: ra = va; break;
          case 1: ra.x = va.y; ra.y = -va.x; break;
          case 2: ra.x = -va.x; ra.y = -va.y; break;
          default: ra.x = -va.y; ra.y = va.x; break;
        }
        switch (kb & 3) {
          case 0: rb = vb; break;
          case 1: rb.x = vb.y; rb.y = -vb.x; break;
          case 2: rb.x = -vb.x; rb.y = -vb.y; break;
          default: rb.x = -vb.y; rb.y = vb.x; break;
        }
        v = cadd(ra, rb);
      }
      // w_m e^{-i m phi0}
      T wm = (m > 0) ? (T)2 : (T)1;
      if (shifted) {
        // e^{-i pi m2 / N}, m2 = m mod 2N = q (N/2) + r: conj(e^{i pi r / N} i^q)
        const int m2 = m % (2 * N), q = m2 / (N >> 1), rr = m2 - q * (N >> 1);
        const T2 er = rot_ik(eph[rr], q);
        T2 e;
        e.x = wm * er.x;
        e.y = -wm * er.y;
        v = cmul(v, e);
      } else {
        v.x *= wm;
        v.y *= wm;
      }
      if (i0 == 0) {
        F[m] = v;
      } else {
        F[m] = cadd(F[m], v);
      }
    }
    __syncthreads();
  }
}

// Bluestein spectra: one block per non-power-of-two length i; computed in double.
template <typename T>
__global__ void __launch_bounds__(512) bluestein_setup_kernel(int nside, const long long *__restrict__ offset,
                                                              const int *__restrict__ mlen,
                                                              typename RealTraits<T>::T2 *__restrict__ spec,
                                                              const double2 *__restrict__ tw, int TW, int nat_lg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *w = (double2 *)smem_raw;
  const int n = blockIdx.x;
  if (n < 1 || n >= nside + 1) return;
  const long long off = offset[n];
  if (off < 0) return;
  const int M = mlen[n];
  const long long twon = 2LL * n;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    // b_k = conj(chirp) at k in (-n, n), wrapped modulo M
    int kk = (k < n) ? k : (k > M - n ? M - k : -1);
    double2 v = {0.0, 0.0};
    if (kk >= 0) {
      long long q = ((long long)kk * kk) % twon;
      double s, c;
      sincospi((double)q / (double)n, &s, &c);
      v.x = c;
      v.y = -s;
    }
    w[k] = v;
  }
  __syncthreads();
  fft_pow2<double, double2>(w, M, 1, -1, tw, TW);
  typedef typename RealTraits<T>::T2 T2;
  // stored in bit-reversed order, the order in which the shared-memory DIF transform
  // leaves its output, or in natural order for the lengths of the register passes
  const int lgM = 31 - __clz(M);
  const bool nat = nat_lg > 0 && lgM >= nat_lg && lgM <= 12;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const int kr = nat ? k : brev_bits(k, lgM);
    T2 v;
    v.x = (T)(w[kr].x / M);
    v.y = (T)(w[kr].y / M);
    spec[off + k] = v;
  }
  // then the chirp e^{i pi t^2 / n}, t < n
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const long long q = ((long long)t * t) % twon;
    double s, c;
    sincospi((double)q / (double)n, &s, &c);
    T2 v;
    v.x = (T)c;
    v.y = (T)s;
    spec[off + M + t] = v;
  }
}

// Per-ring phase table: for every quarter length ni = 1 .. nside (cap rings of
// nphi = 4 ni, and the belt, ni = nside) the factors e^{i pi t / (4 ni)}, t = 0 .. 2 ni,
// at offset ni^2 - 1 (the tables of ni' < ni take sum (2 ni' + 1) = ni^2 - 1
// entries). They give the class phases of half-pixel-shifted rings and the
// radix-4 twiddles e^{2 pi i p / nphi}; formed in double.
template <typename T>
__global__ void phase_table_kernel(int nside, typename RealTraits<T>::T2 *__restrict__ out) {
  const int ni = blockIdx.x + 1;
  typename RealTraits<T>::T2 *o = out + ((size_t)ni * ni - 1);
  for (int t = threadIdx.x; t <= 2 * ni; t += blockDim.x) {
    double sn, cs;
    sincospi((double)t / (4.0 * ni), &sn, &cs);
    o[t].x = (T)cs;
    o[t].y = (T)sn;
  }
}

size_t phase_table_entries(int nside) { return (size_t)(nside + 1) * (nside + 1) - 1; }

cudaError_t launch_phase_table(const tl_plan *p, void *out, cudaStream_t s) {
  if (p->precision == TL_FP64)
    phase_table_kernel<double><<<p->nside, 256, 0, s>>>(p->nside, (double2 *)out);
  else
    phase_table_kernel<float><<<p->nside, 256, 0, s>>>(p->nside, (float2 *)out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------

// Shared memory of a ring-FFT launch: the ring (4 ni entries) plus a work area for
// the folding partial sums (2 x 512, only when a ring has fewer than 512 classes)
// and, for Bluestein lengths, `batch` sub-transforms of length M.
// Bluestein groups of the register passes: single precision, M from 2^blue_reg_lg up to 2^12
static bool group_reg_blue(const tl_plan *p, const FftGroup &g) {
  if (p->precision == TL_FP64 || p->blue_reg_lg == 0 || g.M == 0) return false;
  const int lgM = 31 - __builtin_clz((unsigned)g.M);
  return lgM >= p->blue_reg_lg && lgM <= 12;
}
// threads of a group's CTA (ring_threads of its kernel instance)
static int group_threads(const tl_plan *p, const FftGroup &g) {
  return (group_reg_blue(p, g) && g.M >= 2048) ? 256 : 512;
}
// threads: the CTA size of the kernel that runs the group (group_threads for the
// forward kernels; 512 for the adjoint), which sets how many register Bluestein
// sub-transforms run at once, each with its own exchange array
static size_t group_smem(const tl_plan *p, const FftGroup &g, int batch, int threads) {
  const size_t e2 = (p->precision == TL_FP64) ? 16 : 8;
  const size_t fold = (2 * g.ni_min + 1 < 512) ? 1024 : 0;
  if (group_reg_blue(p, g)) {  // Y, then one padded exchange array per concurrent sub-transform
    const size_t k = (size_t)threads / ((size_t)g.M / 16);
    size_t wl = (k < 4 ? k : 4) * ((size_t)g.M + (size_t)g.M / 16);
    if (wl < fold) wl = fold;
    return e2 * ((size_t)4 * ring_sub_stride_max(g) + wl);
  }
  size_t wl = g.M ? (size_t)batch * (size_t)g.M : 0;
  if (wl < fold) wl = fold;
  return e2 * ((size_t)4 * ring_sub_stride_max(g) + wl);
}
// Four sub-transforms at once when two CTAs still fit on an SM (or when asked to and
// one fits); one at a time otherwise.
static int group_batch(const tl_plan *p, const FftGroup &g) {
  if (g.M == 0 || p->fft_batch == 1 || group_reg_blue(p, g)) return 1;
  const size_t s4 = group_smem(p, g, 4, 512);
  if (p->fft_batch == 4) return s4 <= 227 * 1024 ? 4 : 1;
  return s4 <= 113 * 1024 ? 4 : 1;
}
// Upper bound over all rings (plan feasibility check): batch 1.
size_t ringfft_smem_bytes(const tl_plan *p) {
  const size_t e2 = (p->precision == TL_FP64) ? 16 : 8;
  size_t wl = (size_t)p->blue_maxm;
  if (wl < 1024) wl = 1024;
  return e2 * ((size_t)4 * ((size_t)p->nside + 16) + wl);
}

template <typename K>
static cudaError_t set_group_smem(const tl_plan *p, K kernel) {
  size_t mx = 0;
  for (int i = 0; i < p->fft_ngroups; ++i) {
    const size_t sm = group_smem(p, p->fft_groups[i], group_batch(p, p->fft_groups[i]), 512);
    if (sm > mx) mx = sm;
  }
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
}

template <typename T>
using RingKernel = void (*)(RingTable, int, int, JobList, BluesteinTable, const typename RealTraits<T>::T2 *, int,
                            int, T, const int *, const typename RealTraits<T>::T2 *);

// The kernel instance of a ring group: single precision has compile-time lengths for
// the belt (sub-transforms of 2^8 .. 2^11, Nside 256 .. 2048) and the larger Bluestein
// groups (M = 2^9 .. 2^12); every other group, and double precision, the generic one.
template <typename T>
static RingKernel<T> pick_ring_kernel(const tl_plan *p, const FftGroup &g) {
  if constexpr (sizeof(T) == 4) {
    const int lgM = g.M ? 31 - __builtin_clz((unsigned)g.M) : 0;
    const int lgn = (g.ni_min == g.ni_max && g.ni_min > 0) ? 31 - __builtin_clz((unsigned)g.ni_min) : 0;
    if (g.M && group_reg_blue(p, g)) {
      switch (lgM) {
        case 11: return ringfft_kernel<T, true, 11, true>;
        case 12: return ringfft_kernel<T, true, 12, true>;
        default: break;
      }
    }
    if (g.M) {
      switch (lgM) {
        case 9: return ringfft_kernel<T, true, 9>;
        case 10: return ringfft_kernel<T, true, 10>;
        case 11: return ringfft_kernel<T, true, 11>;
        case 12: return ringfft_kernel<T, true, 12>;
        default: break;
      }
    } else if (lgn && (1 << lgn) == g.ni_min) {
      switch (lgn) {
        case 8: return ringfft_kernel<T, false, 8>;
        case 9: return ringfft_kernel<T, false, 9>;
        case 10: return ringfft_kernel<T, false, 10>;
        case 11: return ringfft_kernel<T, false, 11>;
        default: break;
      }
    }
  }
  return g.M ? ringfft_kernel<T, true, 0> : ringfft_kernel<T, false, 0>;
}

// Raise a kernel's dynamic shared-memory limit on the current device to what a launch
// needs, once (kept per kernel and device; host-side, not thread-safe, as the rest
// of a plan's launches).
static cudaError_t raise_smem(const void *fn, size_t bytes) {
  constexpr int kMax = 128;
  static const void *keys[kMax];
  static int devs[kMax];
  static size_t vals[kMax];
  static int nk = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int i = 0;
  while (i < nk && (keys[i] != fn || devs[i] != dev)) ++i;
  if (i < nk && vals[i] >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  if (i == nk && nk < kMax) {
    keys[nk] = fn;
    devs[nk] = dev;
    ++nk;
  }
  if (i < kMax) vals[i] = bytes;
  return cudaSuccess;
}

// The register-pass kernel of a ring group, or nullptr: single precision, rings of
// one power-of-two length N = 4 ni = 2^LG (LG 10 .. 13) without aliasing (N > mmax),
// and a twiddle table that reaches W_N.
typedef void (*RegRingKernel)(RingTable, int, JobList, const float2 *, int, float, const int *, const float2 *);
static RegRingKernel pick_reg_kernel(const tl_plan *p, const FftGroup &g, int *lg) {
  if (p->precision == TL_FP64 || !p->ring_reg || g.M != 0 || g.ni_min != g.ni_max) return nullptr;
  const int N = 4 * g.ni_min;
  if ((N & (N - 1)) != 0 || N <= p->mmax || N > p->tw_len) return nullptr;
  // every ring of the group starts a 256-pixel tile of the derivative maps: north cap
  // rings at 2 i (i - 1), south ones at Npix - 2 i (i + 1), belt rings at
  // 2 N (N - 1) + k 4 N (N = nside)
  const long long i = g.ni_min, ns = p->nside, T = kD3Tile;
  const bool aligned = (i == ns) ? ((2 * ns * (ns - 1)) % T == 0 && (4 * ns) % T == 0)
                                 : ((2 * i * (i - 1)) % T == 0 && (p->npix - 2 * i * (i + 1)) % T == 0);
  if (!aligned) return nullptr;
  *lg = 31 - __builtin_clz((unsigned)N);
  switch (*lg) {
    case 10: return ringfft_reg_kernel<10>;
    case 11: return ringfft_reg_kernel<11>;
    case 12: return ringfft_reg_kernel<12>;
    case 13: return ringfft_reg_kernel<13>;
    default: return nullptr;
  }
}

template <typename T>
static cudaError_t ringfft_t(const tl_plan *p, const void *const *planes, const MapJob *jobs, int njobs,
                             cudaStream_t s) {
  JobList jl;
  if (njobs > TL_MAX_JOBS) return cudaErrorInvalidValue;
  jl.n = njobs;
  for (int i = 0; i < njobs; ++i) {
    if (jobs[i].plane < 0 || jobs[i].plane > 3) return cudaErrorInvalidValue;
    const size_t plane_len = (size_t)(jobs[i].il ? d7_rows_il(p->nrings) : p->nrings) * (p->mmax + 1);
    jl.job[i].in = (const typename RealTraits<T>::T2 *)planes[jobs[i].plane] + (size_t)jobs[i].j * plane_len;
    jl.job[i].il = jobs[i].il;
    jl.job[i].k = jobs[i].k;
    jl.job[i].div_sint = jobs[i].div_sint;
    jl.job[i].scale = jobs[i].scale;
    jl.job[i].scalef = (float)jobs[i].scale;
    jl.job[i].out = jobs[i].out;
    jl.job[i].tile = jobs[i].tile;
  }
  const int lgtw = 31 - __builtin_clz((unsigned)p->tw_len);
  for (int gi = 0; gi < p->fft_ngroups; ++gi) {
    const FftGroup &g = p->fft_groups[gi];
    dim3 grid(g.count, (njobs + 1) / 2);
    int lg = 0;
    const RegRingKernel rk = (sizeof(T) == 4) ? pick_reg_kernel(p, g, &lg) : nullptr;
    if (rk) {
      const size_t smem = sizeof(float2) * (size_t)((1 << lg) + (1 << (lg - 4)));
      TL_CUDA_TRY(raise_smem((const void *)rk, smem));
      rk<<<grid, 1 << (lg - 4), smem, s>>>(p->ring, p->mmax, jl, (const float2 *)p->twiddle, lgtw,
                                           (float)(1.0 / (double)(p->lmax + 1)), p->fft_rings + g.first,
                                           (const float2 *)p->phase);
      continue;
    }
    const int batch = group_batch(p, g);
    const RingKernel<T> kern = pick_ring_kernel<T>(p, g);
    const int nt = group_threads(p, g);
    TL_CUDA_TRY(raise_smem((const void *)kern, group_smem(p, g, batch, nt)));
    kern<<<grid, nt, group_smem(p, g, batch, nt), s>>>(
        p->ring, p->nside, p->mmax, jl, p->blue,
        (const typename RealTraits<T>::T2 *)p->twiddle, p->tw_len, batch, (T)(1.0 / (double)(p->lmax + 1)),
        p->fft_rings + g.first, (const typename RealTraits<T>::T2 *)p->phase);
  }
  return cudaGetLastError();
}

cudaError_t launch_ringfft_planes(const tl_plan *p, const void *const *planes, const MapJob *jobs, int njobs,
                                  cudaStream_t s) {
  return p->precision == TL_FP64 ? ringfft_t<double>(p, planes, jobs, njobs, s)
                                 : ringfft_t<float>(p, planes, jobs, njobs, s);
}

cudaError_t launch_ringfft(const tl_plan *p, const MapJob *jobs, int njobs, int, cudaStream_t s) {
  const void *planes[4] = {p->d7_T, p->d7_Q, p->d7_U, p->d7_P};
  return launch_ringfft_planes(p, planes, jobs, njobs, s);
}

template <typename T>
static cudaError_t ringfft_adj_t(const tl_plan *p, void *const *planes, const AdjMapJob *jobs, int njobs,
                                 cudaStream_t s) {
  if (njobs > TL_MAX_ADJ_JOBS) return cudaErrorInvalidValue;
  if (njobs == 0) return cudaSuccess;
  AdjJobList jl;
  jl.n = njobs;
  const size_t plane_len = (size_t)p->nrings * (p->mmax + 1);
  for (int i = 0; i < njobs; ++i) {
    if (jobs[i].plane < 0 || jobs[i].plane > 3) return cudaErrorInvalidValue;
    jl.job[i].base = jobs[i].in;
    jl.job[i].fout = (typename RealTraits<T>::T2 *)planes[jobs[i].plane] + (size_t)jobs[i].j * plane_len;
    jl.job[i].plane = jobs[i].plane;
    jl.job[i].j = jobs[i].j;
    jl.job[i].nk = jobs[i].nk;
    jl.job[i].pad = 0;
  }
  TL_CUDA_TRY(set_group_smem(p, ringfft_adj_kernel<T>));
  for (int gi = 0; gi < p->fft_ngroups; ++gi) {
    const FftGroup &g = p->fft_groups[gi];
    const int batch = group_batch(p, g);
    dim3 grid(g.count, njobs);
    ringfft_adj_kernel<T><<<grid, 512, group_smem(p, g, batch, 512), s>>>(
        p->ring, p->mmax, p->npix, p->nmaps, jl, p->blue,
        (const typename RealTraits<T>::T2 *)p->twiddle, p->tw_len, batch, (double)(p->lmax + 1),
        p->fft_rings + g.first, (const typename RealTraits<T>::T2 *)p->phase, p->blue_reg_lg);
  }
  return cudaGetLastError();
}

cudaError_t launch_ringfft_adjoint(const tl_plan *p, void *const *planes, const AdjMapJob *jobs, int njobs,
                                   cudaStream_t s) {
  return p->precision == TL_FP64 ? ringfft_adj_t<double>(p, planes, jobs, njobs, s)
                                 : ringfft_adj_t<float>(p, planes, jobs, njobs, s);
}

// double-precision twiddles for the setup kernel live in a temporary buffer
cudaError_t launch_bluestein_setup_impl(tl_plan *p, const double2 *tw64, cudaStream_t s) {
  if (p->blue_maxm == 0) return cudaSuccess;
  size_t smem = 16 * (size_t)(p->blue_maxm);
  if (p->precision == TL_FP64) {
    TL_CUDA_TRY(cudaFuncSetAttribute(bluestein_setup_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    bluestein_setup_kernel<double><<<p->nside + 1, 512, smem, s>>>(p->nside, p->blue.offset, p->blue.mlen,
                                                                   (double2 *)p->blue.spec, tw64, p->tw_len,
                                                                   p->blue_reg_lg);
  } else {
    TL_CUDA_TRY(cudaFuncSetAttribute(bluestein_setup_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    bluestein_setup_kernel<float><<<p->nside + 1, 512, smem, s>>>(p->nside, p->blue.offset, p->blue.mlen,
                                                                  (float2 *)p->blue.spec, tw64, p->tw_len,
                                                                  p->blue_reg_lg);
  }
  return cudaGetLastError();
}

}  // namespace tl
