// Register-resident FFT passes for power-of-two transforms held by a group of
// threads (single precision).
//
// A transform of length N = 2^LG is held by TG = N / 16 threads, sixteen values
// each, in the "natural distribution": thread h holds element h + TG c in slot c.
// The passes are those of a decimation-in-frequency FFT on the index's base-16
// digits, highest digit first, and each runs in registers: pass p splits every
// sub-problem of length L into 16 interleaved ones of length m = L / 16,
//   y_q[j] = W_L^{j q} sum_r x[j + m r] W_16^{r q},   j < m, q < 16,
// with the sixteen-point DFT done as 4 x 4 (W = e^{DIR 2 pi i / L}). A pass stores
// its results to one shared-memory array, where sub-problem Q' = Q + S q holds
// y_q at (Q' m + j); the next pass loads its sixteen inputs from there. When
// log2 N is not a multiple of four the last pass has radix 2, 4 or 8 and every
// thread runs 16 / R of them. The last pass writes nothing: its outputs stay in
// registers, again in the natural distribution (thread h, slot c: X[h + TG c]), so
// the caller stores them where they belong. The shared array is padded by one
// element per sixteen (a -> a + a / 16), which makes every load and store of
// every pass reach sixteen distinct banks per half-warp (checked on the CPU for
// N = 2^8 .. 2^14), and keeps the addresses affine in the slot, so they fold into
// immediate offsets. The ordering of the output needs no bit reversal.
#pragma once

#include "fft.cuh"

namespace tl {

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

// X_k = sum_n a_n e^{DIR 2 pi i n k / 4}, in place
template <int DIR>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
  const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
  const float2 id = DIR > 0 ? f2(-d13.y, d13.x) : f2(d13.y, -d13.x);  // DIR i (a1 - a3)
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, id);
  a3 = csub(d02, id);
}

template <int DIR>
__device__ __forceinline__ void dft2(float2 &a0, float2 &a1) {
  const float2 s = cadd(a0, a1), d = csub(a0, a1);
  a0 = s;
  a1 = d;
}

// a e^{DIR 2 pi i E / 16}
template <int DIR, int E>
__device__ __forceinline__ float2 rot16(float2 a) {
  constexpr float C1 = 0.92387953251128675613f, S1 = 0.38268343236508977173f, H = 0.70710678118654752440f;
  if constexpr (E == 0) {
    return a;
  } else if constexpr (E == 4) {
    return DIR > 0 ? f2(-a.y, a.x) : f2(a.y, -a.x);
  } else if constexpr (E == 2) {
    return DIR > 0 ? f2(H * (a.x - a.y), H * (a.x + a.y)) : f2(H * (a.x + a.y), H * (a.y - a.x));
  } else if constexpr (E == 6) {
    return DIR > 0 ? f2(-H * (a.x + a.y), H * (a.x - a.y)) : f2(H * (a.y - a.x), -H * (a.x + a.y));
  } else {
    constexpr float c = (E == 1) ? C1 : (E == 3) ? S1 : -C1;  // E = 1, 3, 9
    constexpr float s0 = (E == 1) ? S1 : (E == 3) ? C1 : -S1;
    constexpr float s = DIR > 0 ? s0 : -s0;
    return f2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
  }
}

// sixteen-point DFT in place, natural order in and out: n = c0 + 4 c1, k = k1 + 4 k2
template <int DIR>
__device__ __forceinline__ void dft16(float2 (&x)[16]) {
#pragma unroll
  for (int c0 = 0; c0 < 4; ++c0) dft4<DIR>(x[c0], x[c0 + 4], x[c0 + 8], x[c0 + 12]);
  x[5] = rot16<DIR, 1>(x[5]);
  x[9] = rot16<DIR, 2>(x[9]);
  x[13] = rot16<DIR, 3>(x[13]);
  x[6] = rot16<DIR, 2>(x[6]);
  x[10] = rot16<DIR, 4>(x[10]);
  x[14] = rot16<DIR, 6>(x[14]);
  x[7] = rot16<DIR, 3>(x[7]);
  x[11] = rot16<DIR, 6>(x[11]);
  x[15] = rot16<DIR, 9>(x[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<DIR>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
  // X[k1 + 4 k2] sits at x[4 k1 + k2]: transpose the 4 x 4 register block
  float2 t;
  t = x[1]; x[1] = x[4]; x[4] = t;
  t = x[2]; x[2] = x[8]; x[8] = t;
  t = x[3]; x[3] = x[12]; x[12] = t;
  t = x[6]; x[6] = x[9]; x[9] = t;
  t = x[7]; x[7] = x[13]; x[13] = t;
  t = x[11]; x[11] = x[14]; x[14] = t;
}

// eight-point DFT in place on a[0..7], natural order: n = c0 + 2 c1, k = k1 + 4 k2
template <int DIR>
__device__ __forceinline__ void dft8(float2 *a) {
  dft4<DIR>(a[0], a[2], a[4], a[6]);
  dft4<DIR>(a[1], a[3], a[5], a[7]);
  a[3] = rot16<DIR, 2>(a[3]);
  a[5] = rot16<DIR, 4>(a[5]);
  a[7] = rot16<DIR, 6>(a[7]);
  dft2<DIR>(a[0], a[1]);
  dft2<DIR>(a[2], a[3]);
  dft2<DIR>(a[4], a[5]);
  dft2<DIR>(a[6], a[7]);
  // X[k1 + 4 k2] at a[2 k1 + k2]
  float2 t0 = a[1], t2 = a[2], t3 = a[3], t4 = a[4], t5 = a[5], t6 = a[6];
  a[1] = t2;  // X1 = a[2]
  a[2] = t4;  // X2 = a[4]
  a[3] = t6;  // X3 = a[6]
  a[4] = t0;  // X4 = a[1]
  a[5] = t3;  // X5 = a[3]
  a[6] = t5;  // X6 = a[5]
}

template <int DIR, int R>
__device__ __forceinline__ void dft_small(float2 *a) {
  if constexpr (R == 2) dft2<DIR>(a[0], a[1]);
  else if constexpr (R == 4) dft4<DIR>(a[0], a[1], a[2], a[3]);
  else dft8<DIR>(a);
}

__device__ __forceinline__ int rpad(int a) { return a + (a >> 4); }
__device__ __forceinline__ float2 conj_if(float2 a, bool c) { return c ? f2(a.x, -a.y) : a; }

template <int LG, int DIR>
struct RegFft {
  static constexpr int N = 1 << LG, TG = N >> 4;
  static constexpr int NP16 = LG >> 2;             // radix-16 passes
  static constexpr int RL = 1 << (LG & 3);         // radix of a shorter last pass (1: none)
  static constexpr int NPASS = NP16 + (RL > 1 ? 1 : 0);
  static constexpr int SMEM = N + (N >> 4);        // padded elements of the exchange array
  static_assert(LG >= 8, "at least two radix-16 passes");

  // y_q *= W_L^{j q}, q = 1..15 (tw[k] = e^{-2 pi i k / TW}, k < TW / 2): four table
  // values (j, 2j, 4j, 8j) and products of at most three of them
  __device__ static void twiddle(float2 (&x)[16], int j, int lgL, const float2 *__restrict__ tw, int lgtw) {
    const int s = j << (lgtw - lgL);
    const bool cj = DIR > 0;
    const float2 w1 = conj_if(__ldg(tw + s), cj), w2 = conj_if(__ldg(tw + 2 * s), cj);
    const float2 w4 = conj_if(__ldg(tw + 4 * s), cj), w8 = conj_if(__ldg(tw + 8 * s), cj);
    const float2 w3 = cmul(w1, w2), w5 = cmul(w1, w4), w6 = cmul(w2, w4), w7 = cmul(w3, w4);
    x[1] = cmul(x[1], w1);
    x[2] = cmul(x[2], w2);
    x[3] = cmul(x[3], w3);
    x[4] = cmul(x[4], w4);
    x[5] = cmul(x[5], w5);
    x[6] = cmul(x[6], w6);
    x[7] = cmul(x[7], w7);
    x[8] = cmul(x[8], w8);
    x[9] = cmul(x[9], cmul(w1, w8));
    x[10] = cmul(x[10], cmul(w2, w8));
    x[11] = cmul(x[11], cmul(w3, w8));
    x[12] = cmul(x[12], cmul(w4, w8));
    x[13] = cmul(x[13], cmul(w5, w8));
    x[14] = cmul(x[14], cmul(w6, w8));
    x[15] = cmul(x[15], cmul(w7, w8));
  }

  template <int P>
  __device__ static void pass(float2 (&x)[16], float2 *sm, int h, const float2 *__restrict__ tw, int lgtw) {
    constexpr bool R16 = P < NP16;
    constexpr int lgR = R16 ? 4 : (LG & 3);
    constexpr int R = 1 << lgR;
    constexpr int lgL = LG - 4 * P;
    constexpr int L = 1 << lgL;
    constexpr int lgm = lgL - lgR;
    constexpr int m = 1 << lgm;
    constexpr int S = 1 << (4 * P);
    constexpr int G = 16 / R;
    constexpr bool LAST = P == NPASS - 1;
    if constexpr (P > 0) {
#pragma unroll
      for (int gi = 0; gi < G; ++gi) {
        const int u = h + TG * gi;
        const int j = u & (m - 1), Q = u >> lgm;
        const int base = Q * L + j;
        if constexpr (m >= 16) {
          const int pb = rpad(base);
#pragma unroll
          for (int r = 0; r < R; ++r) x[gi * R + r] = sm[pb + r * (m + (m >> 4))];
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) x[gi * R + r] = sm[rpad(base + m * r)];
        }
      }
      __syncthreads();  // every input is in registers: the array may be overwritten
    }
    if constexpr (R == 16) {
      dft16<DIR>(x);
    } else {
#pragma unroll
      for (int gi = 0; gi < G; ++gi) dft_small<DIR, R>(x + gi * R);
    }
    if constexpr (!LAST) {
      static_assert(G == 1, "only the last pass may be shorter");
      const int j = h & (m - 1), Q = h >> lgm;
      twiddle(x, j, lgL, tw, lgtw);
      if constexpr (P == 0) __syncthreads();  // the array's previous readers are done
      const int pb = rpad(Q * m + j);
      constexpr int st = S * m + ((S * m) >> 4);  // S m is a multiple of 16
      static_assert((S * m) % 16 == 0, "affine store offsets");
#pragma unroll
      for (int q = 0; q < 16; ++q) sm[pb + q * st] = x[q];
      __syncthreads();
    } else if constexpr (G > 1) {
      // group gi's output q is X[h + TG (gi + G q)]: slot gi + G q
      float2 y[16];
#pragma unroll
      for (int gi = 0; gi < G; ++gi)
#pragma unroll
        for (int q = 0; q < R; ++q) y[gi + G * q] = x[gi * R + q];
#pragma unroll
      for (int c = 0; c < 16; ++c) x[c] = y[c];
    }
  }

  // The whole transform: x holds element h + TG c in slot c on entry and X[h + TG c]
  // on return; sm: SMEM elements (16-byte aligned) that only this group uses. Every
  // thread of the block must call it (it synchronises the block).
  __device__ static void run(float2 (&x)[16], float2 *sm, int h, const float2 *__restrict__ tw, int lgtw) {
    pass<0>(x, sm, h, tw, lgtw);
    if constexpr (NPASS > 1) pass<1>(x, sm, h, tw, lgtw);
    if constexpr (NPASS > 2) pass<2>(x, sm, h, tw, lgtw);
    if constexpr (NPASS > 3) pass<3>(x, sm, h, tw, lgtw);
    if constexpr (NPASS > 4) pass<4>(x, sm, h, tw, lgtw);
    static_assert(NPASS <= 5, "up to 2^18");
  }
};

}  // namespace tl
