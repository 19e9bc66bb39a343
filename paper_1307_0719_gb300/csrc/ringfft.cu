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

// In-place radix-2 DIT FFT on `batch` contiguous arrays of length n (power of two)
// in shared memory. dir = -1: sum x e^{-2 pi i k t/n}; dir = +1: e^{+...}.
// tw[k] = e^{-2 pi i k / TW}, k < TW/2.
template <typename T2>
__device__ void fft_pow2(T2 *a, int n, int batch, int dir, const T2 *__restrict__ tw, int TW) {
  const int nth = blockDim.x, tid = threadIdx.x;
  if (n <= 1) return;
  const int lg = 31 - __clz(n);
  const int total = n * batch;
  for (int e = tid; e < total; e += nth) {
    int b = e / n, k = e - b * n;
    int r = __brev(k) >> (32 - lg);
    if (k < r) {
      T2 t = a[b * n + k];
      a[b * n + k] = a[b * n + r];
      a[b * n + r] = t;
    }
  }
  __syncthreads();
  const int nbf = (n >> 1) * batch;
  for (int len = 2; len <= n; len <<= 1) {
    const int half = len >> 1;
    const int step = TW / len;
    for (int e = tid; e < nbf; e += nth) {
      int b = e / (n >> 1), q = e - b * (n >> 1);
      int grp = q / half, pos = q - grp * half;
      int i0 = b * n + grp * len + pos, i1 = i0 + half;
      T2 w = tw[pos * step];
      if (dir > 0) w.y = -w.y;
      T2 u = a[i0], v = cmul(a[i1], w);
      a[i0] = cadd(u, v);
      a[i1] = csub(u, v);
    }
    __syncthreads();
  }
}

// Bluestein: y_p = sum_{t<n} y_t e^{+2 pi i t p / n} in place, n arbitrary,
// using work[M] and the tabulated spectrum bh = DFT_M(conj chirp) / M.
template <typename T, typename T2>
__device__ void bluestein_inplace(T2 *y, int n, int M, T2 *work, const T2 *__restrict__ bh,
                                  const T2 *__restrict__ tw, int TW) {
  const int nth = blockDim.x, tid = threadIdx.x;
  const long long twon = 2LL * n;
  for (int t = tid; t < M; t += nth) {
    T2 v;
    if (t < n) {
      long long q = ((long long)t * t) % twon;  // chirp e^{i pi t^2 / n}
      T s, c;
      sincos_pi<T>((T)q / (T)n, &s, &c);
      T2 w;
      w.x = c;
      w.y = s;
      v = cmul(y[t], w);
    } else {
      v.x = (T)0;
      v.y = (T)0;
    }
    work[t] = v;
  }
  __syncthreads();
  fft_pow2<T2>(work, M, 1, -1, tw, TW);
  for (int k = tid; k < M; k += nth) work[k] = cmul(work[k], bh[k]);
  __syncthreads();
  fft_pow2<T2>(work, M, 1, +1, tw, TW);
  for (int p = tid; p < n; p += nth) {
    long long q = ((long long)p * p) % twon;
    T s, c;
    sincos_pi<T>((T)q / (T)n, &s, &c);
    T2 w;
    w.x = c;
    w.y = s;
    y[p] = cmul(work[p], w);
  }
  __syncthreads();
}

struct JobDev {
  int plane, j, k, div_sint;
  double scale;
  void *out;
};
#define TL_MAX_JOBS 96
struct JobList {
  int n;
  JobDev job[TL_MAX_JOBS];
};
struct PlaneSet {
  const void *base[4];  // T, Q, U, phi planes: [j][ring][m]
};

// G_m contribution of one job at coefficient m (times e^{i m phi0} and weight).
template <typename T, typename T2>
__device__ __forceinline__ T2 g_term(const T2 *__restrict__ F, int m, int k, T invL, T phase_den, T w0) {
  T2 f = F[m];
  // (i m / L)^k
  T mk = (T)1;
  T mm = (T)m * invL;
  for (int q = 0; q < k; ++q) mk *= mm;
  T2 g;
  switch (k & 3) {
    case 0: g.x = f.x * mk; g.y = f.y * mk; break;
    case 1: g.x = -f.y * mk; g.y = f.x * mk; break;
    case 2: g.x = -f.x * mk; g.y = -f.y * mk; break;
    default: g.x = f.y * mk; g.y = -f.x * mk; break;
  }
  // e^{i m phi0} = e^{i pi m / phase_den} on shifted rings (phase_den = 0: phi0 = 0)
  T w = (m == 0) ? w0 : (T)2 * w0;
  if (phase_den != (T)0) {
    int den = (int)phase_den;
    int q = m % (2 * den);
    T s, c;
    sincos_pi<T>((T)q / phase_den, &s, &c);
    T2 e;
    e.x = c;
    e.y = s;
    g = cmul(g, e);
  }
  g.x *= w;
  g.y *= w;
  return g;
}

template <typename T>
__global__ void __launch_bounds__(512) ringfft_kernel(RingTable rt, int nside, int mmax, int nrings, PlaneSet ps,
                                                      int plane_len, JobList jobs, BluesteinTable bt,
                                                      const typename RealTraits<T>::T2 *__restrict__ tw, int TW,
                                                      int wlen, double invL_d) {
  typedef typename RealTraits<T>::T2 T2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = blockIdx.x;
  const int pair = blockIdx.y;
  const int ja = 2 * pair, jb = 2 * pair + 1;
  const bool hasb = jb < jobs.n;
  const int N = rt.nphi[r];
  const int ni = N >> 2;
  const long long first = rt.first[r];
  const T invL = (T)invL_d;
  const int nth = blockDim.x, tid = threadIdx.x;
  T2 *Y = (T2 *)smem_raw;  // [4][ni], decimated order
  T2 *W = Y + N;           // [wlen] work
  // shifted rings: phi0 = pi / (4 inorth) for caps, pi/(4N) for shifted belt rings
  // half-pixel-shifted rings have phi0 = pi / (4 ni): e^{i m phi0} = e^{i pi m / (4 ni)}
  const T phase_den = (rt.phi0[r] == 0.0) ? (T)0 : (T)(4 * ni);

  const JobDev JA = jobs.job[ja];
  const JobDev JB = hasb ? jobs.job[jb] : jobs.job[ja];
  const T2 *FA = (const T2 *)ps.base[JA.plane] + (size_t)JA.j * plane_len + (size_t)r * (mmax + 1);
  const T2 *FB = (const T2 *)ps.base[JB.plane] + (size_t)JB.j * plane_len + (size_t)r * (mmax + 1);
  // both packed maps are transformed in the normalised units of the Legendre stage
  // (similar magnitudes, so the shared transform's rounding does not leak from a
  // large map into a small one); each job's scale is applied on output
  const T wa = (T)(JA.div_sint ? 1.0 / rt.sint[r] : 1.0);
  const T wb = hasb ? (T)(JB.div_sint ? 1.0 / rt.sint[r] : 1.0) : (T)0;
  const T sa = (T)JA.scale, sb = (T)JB.scale;

  // ---- fold m modulo N into the Hermitian spectrum Z_t, stored at Y[(t%4)*ni + t/4]
  // chunks: C threads share one residue class when N < nth
  const int C = (N >= nth) ? 1 : nth / N;
  if (C == 1) {
    for (int t = tid; t < N; t += nth) {
      const int tm = (N - t) % N;
      T2 Ba = {0, 0}, Bam = {0, 0}, Bb = {0, 0}, Bbm = {0, 0};
      for (int m = t; m <= mmax; m += N) {
        Ba = cadd(Ba, g_term<T, T2>(FA, m, JA.k, invL, phase_den, wa));
        if (hasb) Bb = cadd(Bb, g_term<T, T2>(FB, m, JB.k, invL, phase_den, wb));
      }
      for (int m = tm; m <= mmax; m += N) {
        Bam = cadd(Bam, g_term<T, T2>(FA, m, JA.k, invL, phase_den, wa));
        if (hasb) Bbm = cadd(Bbm, g_term<T, T2>(FB, m, JB.k, invL, phase_den, wb));
      }
      // Z = (Ba + conj(Bam))/2 + i (Bb + conj(Bbm))/2
      T2 z;
      z.x = (T)0.5 * (Ba.x + Bam.x) - (T)0.5 * (Bb.y - Bbm.y);
      z.y = (T)0.5 * (Ba.y - Bam.y) + (T)0.5 * (Bb.x + Bbm.x);
      Y[(t & 3) * ni + (t >> 2)] = z;
    }
  } else {
    // partial sums in W[c * N + t], then a fixed-order reduction (deterministic)
    const int c = tid / N, t = tid - c * N;
    if (c < C) {
      const int tm = (N - t) % N;
      T2 Ba = {0, 0}, Bam = {0, 0}, Bb = {0, 0}, Bbm = {0, 0};
      for (int m = t + c * N; m <= mmax; m += C * N) {
        Ba = cadd(Ba, g_term<T, T2>(FA, m, JA.k, invL, phase_den, wa));
        if (hasb) Bb = cadd(Bb, g_term<T, T2>(FB, m, JB.k, invL, phase_den, wb));
      }
      for (int m = tm + c * N; m <= mmax; m += C * N) {
        Bam = cadd(Bam, g_term<T, T2>(FA, m, JA.k, invL, phase_den, wa));
        if (hasb) Bbm = cadd(Bbm, g_term<T, T2>(FB, m, JB.k, invL, phase_den, wb));
      }
      T2 z;
      z.x = (T)0.5 * (Ba.x + Bam.x) - (T)0.5 * (Bb.y - Bbm.y);
      z.y = (T)0.5 * (Ba.y - Bam.y) + (T)0.5 * (Bb.x + Bbm.x);
      W[c * N + t] = z;
    }
    __syncthreads();
    for (int t2 = tid; t2 < N; t2 += nth) {
      T2 acc = {0, 0};
      for (int cc = 0; cc < C; ++cc) acc = cadd(acc, W[cc * N + t2]);
      Y[(t2 & 3) * ni + (t2 >> 2)] = acc;
    }
  }
  __syncthreads();

  // ---- four length-ni inverse DFTs
  if ((ni & (ni - 1)) == 0) {
    fft_pow2<T2>(Y, ni, 4, +1, tw, TW);
  } else {
    const long long off = bt.offset[ni];
    const int M = bt.mlen[ni];
    const T2 *bh = (const T2 *)bt.spec + off;
    for (int t2 = 0; t2 < 4; ++t2) bluestein_inplace<T, T2>(Y + t2 * ni, ni, M, W, bh, tw, TW);
  }

  // ---- radix-4 pass: X_{p1 + ni p2} = sum_t2 i^{t2 p2} e^{2 pi i t2 p1 / N} Y_t2(p1)
  T *outA = (T *)JA.out + first;
  T *outB = hasb ? (T *)JB.out + first : nullptr;
  for (int p1 = tid; p1 < ni; p1 += nth) {
    T2 y[4];
    y[0] = Y[p1];
#pragma unroll
    for (int t2 = 1; t2 < 4; ++t2) {
      T s, c;
      sincos_pi<T>((T)(2 * t2 * p1) / (T)N, &s, &c);
      T2 w;
      w.x = c;
      w.y = s;
      y[t2] = cmul(Y[t2 * ni + p1], w);
    }
    T2 a0 = cadd(y[0], y[2]), a1 = csub(y[0], y[2]);
    T2 b0 = cadd(y[1], y[3]), b1 = csub(y[1], y[3]);
    T2 ib1;  // i * b1
    ib1.x = -b1.y;
    ib1.y = b1.x;
    T2 X0 = cadd(a0, b0), X2 = csub(a0, b0);
    T2 X1 = cadd(a1, ib1), X3 = csub(a1, ib1);
    outA[p1] = sa * X0.x;
    outA[p1 + ni] = sa * X1.x;
    outA[p1 + 2 * ni] = sa * X2.x;
    outA[p1 + 3 * ni] = sa * X3.x;
    if (hasb) {
      outB[p1] = sb * X0.y;
      outB[p1 + ni] = sb * X1.y;
      outB[p1 + 2 * ni] = sb * X2.y;
      outB[p1 + 3 * ni] = sb * X3.y;
    }
  }
}

// Bluestein spectra: one block per non-power-of-two length i; computed in double.
template <typename T>
__global__ void __launch_bounds__(512) bluestein_setup_kernel(int nside, const long long *__restrict__ offset,
                                                              const int *__restrict__ mlen,
                                                              typename RealTraits<T>::T2 *__restrict__ spec,
                                                              const double2 *__restrict__ tw, int TW) {
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
  fft_pow2<double2>(w, M, 1, -1, tw, TW);
  typedef typename RealTraits<T>::T2 T2;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    T2 v;
    v.x = (T)(w[k].x / M);
    v.y = (T)(w[k].y / M);
    spec[off + k] = v;
  }
}

// ---------------------------------------------------------------------------

// shared memory of the ring FFT: the ring (<= 4 nside) plus a work area that
// holds the largest Bluestein transform or the folding partial sums (512)
size_t ringfft_smem_bytes(const tl_plan *p) {
  size_t e2 = (p->precision == TL_FP64) ? 16 : 8;
  int wl = p->blue_maxm > 512 ? p->blue_maxm : 512;
  return e2 * (size_t)(4 * p->nside + wl);
}

template <typename T>
static cudaError_t ringfft_t(const tl_plan *p, const MapJob *jobs, int njobs, cudaStream_t s) {
  JobList jl;
  if (njobs > TL_MAX_JOBS) return cudaErrorInvalidValue;
  jl.n = njobs;
  for (int i = 0; i < njobs; ++i) {
    jl.job[i].plane = jobs[i].plane;
    jl.job[i].j = jobs[i].j;
    jl.job[i].k = jobs[i].k;
    jl.job[i].div_sint = jobs[i].div_sint;
    jl.job[i].scale = jobs[i].scale;
    jl.job[i].out = jobs[i].out;
  }
  PlaneSet ps;
  ps.base[0] = p->d7_T;
  ps.base[1] = p->d7_Q;
  ps.base[2] = p->d7_U;
  ps.base[3] = p->d7_P;
  const int plane_len = p->nrings * (p->mmax + 1);
  size_t smem = ringfft_smem_bytes(p);
  int wlen = (int)(smem / sizeof(typename RealTraits<T>::T2)) - 4 * p->nside;
  TL_CUDA_TRY(cudaFuncSetAttribute(ringfft_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid(p->nrings, (njobs + 1) / 2);
  ringfft_kernel<T><<<grid, 512, smem, s>>>(p->ring, p->nside, p->mmax, p->nrings, ps, plane_len, jl, p->blue,
                                            (const typename RealTraits<T>::T2 *)p->twiddle, p->tw_len, wlen,
                                            1.0 / (double)(p->lmax + 1));
  return cudaGetLastError();
}

cudaError_t launch_ringfft(const tl_plan *p, const MapJob *jobs, int njobs, int, cudaStream_t s) {
  return p->precision == TL_FP64 ? ringfft_t<double>(p, jobs, njobs, s) : ringfft_t<float>(p, jobs, njobs, s);
}

// double-precision twiddles for the setup kernel live in a temporary buffer
cudaError_t launch_bluestein_setup_impl(tl_plan *p, const double2 *tw64, cudaStream_t s) {
  if (p->blue_maxm == 0) return cudaSuccess;
  size_t smem = 16 * (size_t)(p->blue_maxm);
  if (p->precision == TL_FP64) {
    TL_CUDA_TRY(cudaFuncSetAttribute(bluestein_setup_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    bluestein_setup_kernel<double><<<p->nside + 1, 512, smem, s>>>(p->nside, p->blue.offset, p->blue.mlen,
                                                                   (double2 *)p->blue.spec, tw64, p->tw_len);
  } else {
    TL_CUDA_TRY(cudaFuncSetAttribute(bluestein_setup_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    bluestein_setup_kernel<float><<<p->nside + 1, 512, smem, s>>>(p->nside, p->blue.offset, p->blue.mlen,
                                                                  (float2 *)p->blue.spec, tw64, p->tw_len);
  }
  return cudaGetLastError();
}

}  // namespace tl
