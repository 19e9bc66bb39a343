// Shared-memory FFT building blocks used by the ring synthesis and its adjoint:
// complex helpers, an in-place radix-2 FFT over batches of power-of-two arrays,
// and Bluestein's chirp-z transform for other lengths.
#pragma once

#include "legendre.cuh"

namespace tl {

template <typename T> struct C2 {
  typedef typename RealTraits<T>::T2 T2;
};

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  T2 r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename T2>
__device__ __forceinline__ T2 cadd(T2 a, T2 b) {
  T2 r;
  r.x = a.x + b.x;
  r.y = a.y + b.y;
  return r;
}
template <typename T2>
__device__ __forceinline__ T2 csub(T2 a, T2 b) {
  T2 r;
  r.x = a.x - b.x;
  r.y = a.y - b.y;
  return r;
}

template <typename T> __device__ __forceinline__ void sincos_pi(T x, T *s, T *c);
template <> __device__ __forceinline__ void sincos_pi<float>(float x, float *s, float *c) { sincospif(x, s, c); }
template <> __device__ __forceinline__ void sincos_pi<double>(double x, double *s, double *c) { sincospi(x, s, c); }

// Shared-memory layout of power-of-two arrays: element i of array b (length 2^lg)
// sits at b * stride + swz(i, lg) ^ (b & 3). swz XORs bits 4-6, bit 6 and the top
// bits of i into its low four bits (16 banks of 8-byte elements), a bijection within
// every 16-element block, chosen so that the fused FFT passes at every span, the
// bit-reversed writes of the fold and of Bluestein, and the natural-order passes
// all reach distinct banks (checked for lengths up to 2^13: at most 1.5 wavefronts
// per 16 threads, against 16 for a plain or padded layout on bit-reversed writes).
__host__ __device__ __forceinline__ int swz(int i, int lg) {
  const int f1 = (i >> 4) & 7;
  const int f2 = ((i >> 6) & 1) << 3;
  const int f3 = lg >= 8 ? (i >> (lg - 4 > 7 ? lg - 4 : 7)) & 15 : 0;
  return i ^ f1 ^ f2 ^ f3;
}
__host__ __device__ __forceinline__ int faddr(int b, int i, int lg, int stride) {
  return b * stride + (swz(i, lg) ^ (b & 3));
}
__device__ __forceinline__ int brev_bits(int e, int lg) { return lg == 0 ? 0 : (int)(__brev((unsigned)e) >> (32 - lg)); }

// e^{-2 pi i cc / 2^(lev+1)} (conjugated for dir > 0), cc < 2^lev, lev <= 3
template <typename T, typename T2>
__device__ __forceinline__ T2 unit_root(int lev, int cc, int dir) {
  const T h = (T)0.70710678118654752440;
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;  // cos, sin of pi/8
  T2 r;
  if (lev == 1) {
    r.x = (T)0;
    r.y = (T)-1;
  } else if (lev == 2) {
    r.x = (cc == 1) ? h : (cc == 2) ? (T)0 : -h;
    r.y = (cc == 2) ? (T)-1 : -h;
  } else {  // lev == 3: cos and -sin of 2 pi cc / 16
    const T cn = (cc == 0) ? (T)1 : (cc == 1) ? c1 : (cc == 2) ? h : (cc == 3) ? s1 : (cc == 4) ? (T)0
               : (cc == 5) ? -s1 : (cc == 6) ? -h : -c1;
    const T sn = (cc == 0) ? (T)0 : (cc == 1) ? s1 : (cc == 2) ? h : (cc == 3) ? c1 : (cc == 4) ? (T)1
               : (cc == 5) ? c1 : (cc == 6) ? h : s1;
    r.x = cn;
    r.y = -sn;
  }
  if (dir > 0) r.y = -r.y;
  return r;
}

// R consecutive radix-2 DIT stages (half-spans 2^sh .. 2^(sh+R-1)) fused into one
// pass: each thread loads the 2^R elements i0 + c 2^sh of one group, runs the R
// levels of butterflies in registers and stores them back. At stage s an element
// whose bit s is clear pairs with the one 2^s above it, with the twiddle
// W_{2^(s+1)}^(index mod 2^s) = W_{2^(s+1)}^pos W_{2^(lev+1)}^cc: one table load
// per level times a fixed root of unity.
template <int R, bool SWZ, typename T, typename T2, int LGC = 0>
__device__ __forceinline__ void dit_pass(T2 *a, int lg_rt, int batch, int stride, int sh, int dir,
                                         const T2 *__restrict__ tw, int lgtw) {
  const int lg = LGC ? LGC : lg_rt;  // a compile-time length folds the index arithmetic
  constexpr int P = 1 << R;
  const int ulg = lg - R;  // groups per array: 2^ulg
  const int total = batch << ulg;
  const int h = 1 << sh;
  // swz is linear over XOR and i0 has bits sh .. sh+R-1 clear, so the element
  // addresses are faddr(b, i0) ^ swz(c << sh): offsets d[c] shared by every group
  int d[P];
#pragma unroll
  for (int c = 0; c < P; ++c) d[c] = SWZ ? swz(c << sh, lg) : (c << sh);
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int b = e >> ulg, q = e & ((1 << ulg) - 1);
    const int pos = q & (h - 1), grp = q >> sh;
    const int i0 = (grp << (sh + R)) + pos;
    const int base = SWZ ? faddr(b, i0, lg, stride) : b * stride + i0;
    T2 x[P];
#pragma unroll
    for (int c = 0; c < P; ++c) x[c] = a[SWZ ? (base ^ d[c]) : base + d[c]];
#pragma unroll
    for (int lev = 0; lev < R; ++lev) {
      T2 wl = tw[pos << (lgtw - sh - lev - 1)];
      if (dir > 0) wl.y = -wl.y;
#pragma unroll
      for (int c = 0; c < P; ++c) {
        if ((c >> lev) & 1) continue;
        const int cc = c & ((1 << lev) - 1);
        const T2 w = cc ? cmul(wl, unit_root<T, T2>(lev, cc, dir)) : wl;
        const T2 u = x[c], v = cmul(x[c + (1 << lev)], w);
        x[c] = cadd(u, v);
        x[c + (1 << lev)] = csub(u, v);
      }
    }
#pragma unroll
    for (int c = 0; c < P; ++c) a[SWZ ? (base ^ d[c]) : base + d[c]] = x[c];
  }
  __syncthreads();
}

// The top DIT pass of the inverse transform in Bluestein: as dit_pass (dir +1), but
// each output p < n is multiplied by the chirp e^{i pi p^2/n} and written to y;
// the rest (p >= n) are not needed.
template <int R, typename T, typename T2, int LGC = 0>
__device__ __forceinline__ void dit_last(const T2 *a, int lg_rt, int batch, int stride, int sh,
                                         const T2 *__restrict__ tw, int lgtw, T2 *y, int n, int ystride,
                                         const T2 *__restrict__ chirp) {
  const int lg = LGC ? LGC : lg_rt;
  constexpr int P = 1 << R;
  const int ulg = lg - R;
  const int total = batch << ulg;
  const int h = 1 << sh;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int b = e >> ulg, q = e & ((1 << ulg) - 1);
    const int pos = q & (h - 1), grp = q >> sh;
    const int i0 = (grp << (sh + R)) + pos;
    const int base = faddr(b, i0, lg, stride);
    T2 x[P];
#pragma unroll
    for (int c = 0; c < P; ++c) x[c] = a[base ^ swz(c << sh, lg)];
#pragma unroll
    for (int lev = 0; lev < R; ++lev) {
      T2 wl = tw[pos << (lgtw - sh - lev - 1)];
      wl.y = -wl.y;
#pragma unroll
      for (int c = 0; c < P; ++c) {
        if ((c >> lev) & 1) continue;
        const int cc = c & ((1 << lev) - 1);
        const T2 w = cc ? cmul(wl, unit_root<T, T2>(lev, cc, +1)) : wl;
        const T2 u = x[c], v = cmul(x[c + (1 << lev)], w);
        x[c] = cadd(u, v);
        x[c + (1 << lev)] = csub(u, v);
      }
    }
#pragma unroll
    for (int c = 0; c < P; ++c) {
      const int p = i0 + (c << sh);
      if (p < n) y[b * ystride + p] = cmul(x[c], chirp[p]);
    }
  }
  __syncthreads();
}

// In-place DIT FFT on `batch` arrays of length n (power of two), `stride` elements
// apart (swizzled layout when SWZ), whose input is already in bit-reversed order
// (the writers store it so);
// output in natural order. dir = -1: sum x e^{-2 pi i k t/n}; dir = +1: e^{+...}.
// tw[k] = e^{-2 pi i k / TW}, k < TW/2 (TW >= n). Passes of four stages, then the
// remainder. LGC > 0: n = 2^LGC known at compile time (passes unrolled).
template <bool SWZ, typename T, typename T2, int LGC = 0>
__device__ __forceinline__ void fft_core(T2 *a, int n, int batch, int stride, int dir, const T2 *__restrict__ tw,
                                         int TW) {
  const int lg = LGC ? LGC : 31 - __clz(n);
  if (lg == 0) return;
  const int lgtw = 31 - __clz(TW);
  int sh = 0;
#pragma unroll
  for (; sh + 4 <= lg; sh += 4) dit_pass<4, SWZ, T, T2, LGC>(a, lg, batch, stride, sh, dir, tw, lgtw);
  if (lg - sh == 3) dit_pass<3, SWZ, T, T2, LGC>(a, lg, batch, stride, sh, dir, tw, lgtw);
  if (lg - sh == 2) dit_pass<2, SWZ, T, T2, LGC>(a, lg, batch, stride, sh, dir, tw, lgtw);
  if (lg - sh == 1) dit_pass<1, SWZ, T, T2, LGC>(a, lg, batch, stride, sh, dir, tw, lgtw);
}

// The same for contiguous, unpadded arrays in natural order (bit-reversal first).
template <typename T, typename T2>
__device__ void fft_pow2(T2 *a, int n, int batch, int dir, const T2 *__restrict__ tw, int TW) {
  if (n <= 1) return;
  const int lg = 31 - __clz(n);
  for (int e = threadIdx.x; e < n * batch; e += blockDim.x) {
    const int k = e & (n - 1);
    const int r = brev_bits(k, lg);
    if (k < r) {
      const int base = e - k;
      T2 t = a[base + k];
      a[base + k] = a[base + r];
      a[base + r] = t;
    }
  }
  __syncthreads();
  fft_core<false, T, T2>(a, n, batch, n, dir, tw, TW);
}

// R fused radix-2 decimation-in-frequency stages (half-spans 2^(sh+R-1) down to
// 2^sh) on the swizzled work arrays: each thread takes the 2^R elements
// i0 + c 2^sh of one group, and at each level pairs c with c + 2^lev:
// (u, v) -> (u + v, (u - v) W), W = W_{2^(sh+lev+1)}^(index mod 2^(sh+lev)) (the same
// twiddles as dit_pass). DIF takes natural order in; after all passes the output is
// in bit-reversed order.
//   FIRST: the inputs are y_t e^{i pi t^2/n} read from y (t < n, zero from n on;
//          n <= 2^(lg-1), so the upper half of the first level is zero);
//   LAST:  each output is multiplied by the tabulated spectrum (bit-reversed order)
//          as it is stored.
template <int R, bool FIRST, bool LAST, typename T, typename T2, int LGC = 0>
__device__ __forceinline__ void bs_dif_pass(T2 *w, int lg_rt, int batch, int wstride, int sh,
                                            const T2 *__restrict__ tw, int lgtw, const T2 *y, int n, int ystride,
                                            const T2 *__restrict__ chirp, const T2 *__restrict__ bhr) {
  const int lg = LGC ? LGC : lg_rt;
  constexpr int P = 1 << R;
  const int ulg = lg - R;
  const int total = batch << ulg;
  const int h = 1 << sh;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int b = e >> ulg, q = e & ((1 << ulg) - 1);
    const int pos = q & (h - 1), grp = q >> sh;
    const int i0 = (grp << (sh + R)) + pos;
    const int base = faddr(b, i0, lg, wstride);
    T2 x[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      if (FIRST) {
        const int t = i0 + (c << sh);
        T2 v;
        v.x = (T)0;
        v.y = (T)0;
        if (c < P / 2 && t < n) v = cmul(y[b * ystride + t], chirp[t]);
        x[c] = v;
      } else {
        x[c] = w[base ^ swz(c << sh, lg)];
      }
    }
#pragma unroll
    for (int lev = R - 1; lev >= 0; --lev) {
      const T2 wl = tw[pos << (lgtw - sh - lev - 1)];
#pragma unroll
      for (int c = 0; c < P; ++c) {
        if ((c >> lev) & 1) continue;
        const int cc = c & ((1 << lev) - 1);
        const T2 wt = cc ? cmul(wl, unit_root<T, T2>(lev, cc, -1)) : wl;
        const T2 u = x[c], v = x[c + (1 << lev)];
        if (FIRST && lev == R - 1) {  // v is zero (upper half of the first level)
          x[c + (1 << lev)] = cmul(u, wt);
        } else {
          x[c] = cadd(u, v);
          x[c + (1 << lev)] = cmul(csub(u, v), wt);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < P; ++c) {
      const int off = swz(c << sh, lg);
      w[base ^ off] = LAST ? cmul(x[c], bhr[i0 + (c << sh)]) : x[c];
    }
  }
  __syncthreads();
}

// Bluestein on `batch` sequences y (plain layout, ystride apart) of length n (n
// arbitrary), in place: y_p <- sum_{t<n} y_t e^{+2 pi i t p / n}. With
// tp = (t^2 + p^2 - (p-t)^2)/2 the DFT is a chirp, a circular convolution of length
// M >= 2n (powers of two) against the spectrum of the conjugate chirp, and a chirp:
// a forward DIF transform of the chirped input (natural order in, bit-reversed out;
// the chirp applied as its first pass loads), the product with the tabulated
// spectrum bhr (stored in bit-reversed order, 1/M included; applied as the last DIF
// pass stores), the inverse DIT transform (bit-reversed in, natural out), whose last
// pass multiplies by the chirp and writes the n outputs back to y. No bit-reversal
// pass, no scatter: work holds batch swizzled arrays of length M, wstride apart.
template <typename T, typename T2, int LGC = 0>
__device__ __forceinline__ void bluestein_batch(T2 *y, int n, int ystride, int M, int batch, T2 *work, int wstride,
                                                const T2 *__restrict__ bhr, const T2 *__restrict__ chirp,
                                                const T2 *__restrict__ tw, int TW) {
  const int lg = LGC ? LGC : 31 - __clz(M);  // M >= 2n >= 8 for every Bluestein length
  const int lgtw = 31 - __clz(TW);
  // ---- forward DIF: passes of four stages from the top (three when M = 8), then the
  // remainder; the first pass reads the chirped input, the last applies the spectrum
  if (lg < 4) {
    if (lg == 3)
      bs_dif_pass<3, true, true, T, T2, LGC>(work, lg, batch, wstride, 0, tw, lgtw, y, n, ystride, chirp, bhr);
  } else {
    const int r = lg % 4;
    int sh = lg - 4;
    if (sh == 0) {
      bs_dif_pass<4, true, true, T, T2, LGC>(work, lg, batch, wstride, 0, tw, lgtw, y, n, ystride, chirp, bhr);
    } else {
      bs_dif_pass<4, true, false, T, T2, LGC>(work, lg, batch, wstride, sh, tw, lgtw, y, n, ystride, chirp, bhr);
#pragma unroll
      for (sh -= 4; sh >= 0; sh -= 4) {
        if (sh == 0)
          bs_dif_pass<4, false, true, T, T2, LGC>(work, lg, batch, wstride, 0, tw, lgtw, y, n, ystride, chirp, bhr);
        else
          bs_dif_pass<4, false, false, T, T2, LGC>(work, lg, batch, wstride, sh, tw, lgtw, y, n, ystride, chirp,
                                                   bhr);
      }
      if (r == 3)
        bs_dif_pass<3, false, true, T, T2, LGC>(work, lg, batch, wstride, 0, tw, lgtw, y, n, ystride, chirp, bhr);
      if (r == 2)
        bs_dif_pass<2, false, true, T, T2, LGC>(work, lg, batch, wstride, 0, tw, lgtw, y, n, ystride, chirp, bhr);
      if (r == 1)
        bs_dif_pass<1, false, true, T, T2, LGC>(work, lg, batch, wstride, 0, tw, lgtw, y, n, ystride, chirp, bhr);
    }
  }
  // ---- inverse DIT, natural order out: passes of four stages from the bottom; the
  // top pass (the remaining 1 to 4 stages) writes the chirped outputs p < n to y
  int s0 = 0;
#pragma unroll
  for (; s0 + 4 < lg; s0 += 4) dit_pass<4, true, T, T2, LGC>(work, lg, batch, wstride, s0, +1, tw, lgtw);
  const int R = lg - s0;
  if (R == 4) dit_last<4, T, T2, LGC>(work, lg, batch, wstride, s0, tw, lgtw, y, n, ystride, chirp);
  if (R == 3) dit_last<3, T, T2, LGC>(work, lg, batch, wstride, s0, tw, lgtw, y, n, ystride, chirp);
  if (R == 2) dit_last<2, T, T2, LGC>(work, lg, batch, wstride, s0, tw, lgtw, y, n, ystride, chirp);
  if (R == 1) dit_last<1, T, T2, LGC>(work, lg, batch, wstride, s0, tw, lgtw, y, n, ystride, chirp);
}

}  // namespace tl
