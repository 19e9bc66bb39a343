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

// e^{-2 pi i cc / 2^(lev+1)} (conjugated for dir > 0), cc < 2^lev, lev <= 2
template <typename T, typename T2>
__device__ __forceinline__ T2 unit_root(int lev, int cc, int dir) {
  const T h = (T)0.70710678118654752440;
  T2 r;
  if (lev == 1) {
    r.x = (T)0;
    r.y = (T)-1;
  } else {  // lev == 2
    r.x = (cc == 1) ? h : (cc == 2) ? (T)0 : -h;
    r.y = (cc == 2) ? (T)-1 : -h;
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
template <int R, bool SWZ, typename T, typename T2>
__device__ __forceinline__ void dit_pass(T2 *a, int lg, int batch, int stride, int sh, int dir,
                                         const T2 *__restrict__ tw, int lgtw) {
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

// In-place DIT FFT on `batch` arrays of length n (power of two), `stride` elements
// apart (swizzled layout when SWZ), whose input is already in bit-reversed order
// (the writers store it so);
// output in natural order. dir = -1: sum x e^{-2 pi i k t/n}; dir = +1: e^{+...}.
// tw[k] = e^{-2 pi i k / TW}, k < TW/2 (TW >= n). Passes of three stages.
template <bool SWZ, typename T, typename T2>
__device__ void fft_core(T2 *a, int n, int batch, int stride, int dir, const T2 *__restrict__ tw, int TW) {
  if (n <= 1) return;
  const int lg = 31 - __clz(n);
  const int lgtw = 31 - __clz(TW);
  int sh = 0;
  for (; sh + 3 <= lg; sh += 3) dit_pass<3, SWZ, T, T2>(a, lg, batch, stride, sh, dir, tw, lgtw);
  if (lg - sh == 2) dit_pass<2, SWZ, T, T2>(a, lg, batch, stride, sh, dir, tw, lgtw);
  if (lg - sh == 1) dit_pass<1, SWZ, T, T2>(a, lg, batch, stride, sh, dir, tw, lgtw);
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

// Bluestein on `batch` sequences y (plain layout, ystride apart) of length n (n
// arbitrary), in place: y_p <- sum_{t<n} y_t e^{+2 pi i t p / n}. With
// tp = (t^2 + p^2 - (p-t)^2)/2 the DFT is a chirp, a circular convolution of length
// M >= 2n - 1 (two power-of-two FFTs against the tabulated spectrum
// bh = DFT_M(conj chirp) / M) and a chirp. work: batch swizzled arrays of length M,
// wstride apart. Each pass writes the next transform's input in bit-reversed order.
template <typename T, typename T2>
__device__ void bluestein_batch(T2 *y, int n, int ystride, int M, int batch, T2 *work, int wstride,
                                const T2 *__restrict__ bh, const T2 *__restrict__ chirp,
                                const T2 *__restrict__ tw, int TW) {
  const int nth = blockDim.x, tid = threadIdx.x;
  const int lgM = 31 - __clz(M);
  for (int t = tid; t < M; t += nth) {
    const int d = brev_bits(t, lgM);
    if (t < n) {
      const T2 w = chirp[t];  // e^{i pi t^2 / n}
      for (int b = 0; b < batch; ++b) work[faddr(b, d, lgM, wstride)] = cmul(y[b * ystride + t], w);
    } else {
      T2 z;
      z.x = (T)0;
      z.y = (T)0;
      for (int b = 0; b < batch; ++b) work[faddr(b, d, lgM, wstride)] = z;
    }
  }
  __syncthreads();
  fft_core<true, T, T2>(work, M, batch, wstride, -1, tw, TW);
  // multiply by the spectrum, writing bit-reversed for the inverse transform
  for (int k = tid; k < M; k += nth) {
    const int r = brev_bits(k, lgM);
    if (k > r) continue;
    const T2 hk = bh[k], hr = bh[r];
    for (int b = 0; b < batch; ++b) {
      const int ak = faddr(b, k, lgM, wstride), ar = faddr(b, r, lgM, wstride);
      const T2 xk = work[ak], xr = work[ar];
      work[ar] = cmul(xk, hk);
      work[ak] = cmul(xr, hr);
    }
  }
  __syncthreads();
  fft_core<true, T, T2>(work, M, batch, wstride, +1, tw, TW);
  for (int p = tid; p < n; p += nth) {
    const T2 w = chirp[p];
    for (int b = 0; b < batch; ++b) y[b * ystride + p] = cmul(work[faddr(b, p, lgM, wstride)], w);
  }
  __syncthreads();
}

}  // namespace tl
