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

// R consecutive radix-2 DIT stages (half-spans 2^sh .. 2^(sh+R-1)) fused into one
// pass: each thread loads the 2^R elements base + c 2^sh of one group, runs the R
// levels of butterflies in registers and stores them back. At stage s an element
// whose bit s is clear pairs with the one 2^s above it, with the twiddle
// W_{2^(s+1)}^(index mod 2^s).
template <int R, typename T2>
__device__ __forceinline__ void dit_pass(T2 *a, int lg, int batch, int sh, int dir, const T2 *__restrict__ tw,
                                         int lgtw) {
  constexpr int P = 1 << R;
  const int ulg = lg - R;  // groups per array: 2^ulg
  const int total = batch << ulg;
  const int h = 1 << sh;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int b = e >> ulg, q = e & ((1 << ulg) - 1);
    const int pos = q & (h - 1), grp = q >> sh;
    T2 *base = a + (b << lg) + (grp << (sh + R)) + pos;
    T2 x[P];
#pragma unroll
    for (int c = 0; c < P; ++c) x[c] = base[c << sh];
#pragma unroll
    for (int lev = 0; lev < R; ++lev) {
#pragma unroll
      for (int c = 0; c < P; ++c) {
        if ((c >> lev) & 1) continue;
        const int cc = c & ((1 << lev) - 1);
        T2 w = tw[(pos + (cc << sh)) << (lgtw - sh - lev - 1)];
        if (dir > 0) w.y = -w.y;
        const T2 u = x[c], v = cmul(x[c + (1 << lev)], w);
        x[c] = cadd(u, v);
        x[c + (1 << lev)] = csub(u, v);
      }
    }
#pragma unroll
    for (int c = 0; c < P; ++c) base[c << sh] = x[c];
  }
  __syncthreads();
}

// In-place DIT FFT on `batch` contiguous arrays of length n (power of two) in
// shared memory. dir = -1: sum x e^{-2 pi i k t/n}; dir = +1: e^{+...}.
// tw[k] = e^{-2 pi i k / TW}, k < TW/2 (TW >= n). A bit-reversal permutation, then
// the log2 n radix-2 stages in passes of three (eight elements per thread).
template <typename T2>
__device__ void fft_pow2(T2 *a, int n, int batch, int dir, const T2 *__restrict__ tw, int TW) {
  const int nth = blockDim.x, tid = threadIdx.x;
  if (n <= 1) return;
  const int lg = 31 - __clz(n);
  const int total = n * batch;
  for (int e = tid; e < total; e += nth) {
    const int k = e & (n - 1);
    const int r = __brev(k) >> (32 - lg);
    if (k < r) {
      const int base = e - k;
      T2 t = a[base + k];
      a[base + k] = a[base + r];
      a[base + r] = t;
    }
  }
  __syncthreads();
  const int lgtw = 31 - __clz(TW);
  int sh = 0;
  for (; sh + 3 <= lg; sh += 3) dit_pass<3, T2>(a, lg, batch, sh, dir, tw, lgtw);
  if (lg - sh == 2) dit_pass<2, T2>(a, lg, batch, sh, dir, tw, lgtw);
  if (lg - sh == 1) dit_pass<1, T2>(a, lg, batch, sh, dir, tw, lgtw);
}

// Bluestein on `batch` contiguous sequences y[b n + t] of length n (n arbitrary),
// in place: y_p <- sum_{t<n} y_t e^{+2 pi i t p / n}. With tp = (t^2 + p^2 - (p-t)^2)/2
// the DFT is a chirp, a circular convolution of length M >= 2n - 1 (done by two
// power-of-two FFTs against the tabulated spectrum bh = DFT_M(conj chirp) / M)
// and a chirp. work holds batch * M entries.
template <typename T, typename T2>
__device__ void bluestein_batch(T2 *y, int n, int M, int batch, T2 *work, const T2 *__restrict__ bh,
                                const T2 *__restrict__ chirp, const T2 *__restrict__ tw, int TW) {
  const int nth = blockDim.x, tid = threadIdx.x;
  for (int t = tid; t < M; t += nth) {
    if (t < n) {
      const T2 w = chirp[t];  // e^{i pi t^2 / n}
      for (int b = 0; b < batch; ++b) work[b * M + t] = cmul(y[b * n + t], w);
    } else {
      T2 z;
      z.x = (T)0;
      z.y = (T)0;
      for (int b = 0; b < batch; ++b) work[b * M + t] = z;
    }
  }
  __syncthreads();
  fft_pow2<T2>(work, M, batch, -1, tw, TW);
  for (int k = tid; k < M; k += nth) {
    const T2 h = bh[k];
    for (int b = 0; b < batch; ++b) work[b * M + k] = cmul(work[b * M + k], h);
  }
  __syncthreads();
  fft_pow2<T2>(work, M, batch, +1, tw, TW);
  for (int p = tid; p < n; p += nth) {
    const T2 w = chirp[p];
    for (int b = 0; b < batch; ++b) y[b * n + p] = cmul(work[b * M + p], w);
  }
  __syncthreads();
}

}  // namespace tl
