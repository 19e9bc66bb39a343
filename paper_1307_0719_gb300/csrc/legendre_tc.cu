// Legendre stage with the contraction on the tensor cores (Naess & Louis 2013,
// Sec. II.B: the derivative maps of Eq. 4).
//
// The recurrence runs exactly as in legendre.cu (one thread per ring, FP32 with
// FP64 seeds and exponent scaling, normalised step mu_{l+1} = A X mu_l - mu_{l-1},
// theta-derivatives by Leibniz's rule). Every 8 values of l, each warp holds a
// [32 rings x 8 l] tile of mu^(j) per derivative order j; the contraction against
// the coefficient sets is then the dense product
//     D^(j)[rings x N] += Mu^(j)[rings x 8] . C[8 x N]
// done with mma.sync m16n8k8 TF32 (two 16-row tiles per warp). N = 8 columns hold
// the coefficient sets of up to two realisations that share the basis:
//   spin 2: (k_l (E + iB), k_l (-1)^(l+m) (E - iB)) as 4 reals per realisation,
//   spin 0: (k_l a, k_l (-1)^(l+m) a) as 4 reals per realisation (north sum and
//           south parity sum), plus the same for the lensing potential at j <= 1.
// TF32 rounds both operands to 10 mantissa bits; the 3xTF32 form splits each
// operand into hi + lo and accumulates hi.hi + hi.lo + lo.hi (errors near FP32).
// Tiles are staged through shared memory with 16-byte stores and read with
// ldmatrix (the two 16-byte halves of a row swap for rows 4..7 of each 8, which
// makes both the stores and ldmatrix conflict-free).
#include <math.h>
#include <string.h>

#include "legendre.cuh"

namespace tl {

// ---------------------------------------------------------------------------
// helpers

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], uint32_t saddr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(saddr));
}

// byte offset of (row, 16-byte chunk) in a [32 rows][8 floats] tile, halves swapped on rows 4..7 mod 8
__device__ __forceinline__ uint32_t tile_off(int row, int chunk) {
  return (uint32_t)(row * 32 + ((chunk ^ ((row >> 2) & 1)) << 4));
}

// Load the A fragments (rows 0..15 and 16..31) of one [32 x 8] tile.
__device__ __forceinline__ void load_afrag(uint32_t tile_saddr, int lane, uint32_t (&a0)[4], uint32_t (&a1)[4]) {
  const int q = lane >> 3, r = lane & 7;
  const int row = ((q & 1) << 3) + r, chunk = q >> 1;
  ldmatrix_x4(a0, tile_saddr + tile_off(row, chunk));
  ldmatrix_x4(a1, tile_saddr + tile_off(row + 16, chunk));
}

// ---------------------------------------------------------------------------
// plan-time tables: per m, blocks of 8 l starting at l0 = max(m, |s|)

// step factors per block: A_{l+1} (8 floats) then m s/(l(l+1)) (8 floats); 0 past lmax
__global__ void tcstep_kernel(int lmax, int s, const long long *__restrict__ blkofs,
                              const float2 *__restrict__ tab, float *__restrict__ out) {
  const int m = blockIdx.y;
  const int as = s < 0 ? -s : s;
  const int l0 = m > as ? m : as;
  const int nblk = (lmax >= l0) ? (lmax - l0 + 8) / 8 : 0;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;  // (block, slot)
  if (e >= nblk * 8) return;
  const int blk = e >> 3, k = e & 7;
  const int l = l0 + 8 * blk + k;
  float A = 0.0f, ct = 0.0f;
  if (l <= lmax) {
    A = tab[(long long)m * (2 * lmax + 1 - m) / 2 + l].y;
    ct = (float)((double)m * s / ((double)l * (l + 1.0)));
  }
  float *o = out + (blkofs[m] + blk) * 16;
  o[k] = A;
  o[8 + k] = ct;
}

// Coefficient fragments per block: for lane (g, t) the B values at (k = t, n = g)
// and (k = t + 4, n = g), hi and lo TF32 parts: float4 {b0 hi, b1 hi, b0 lo, b1 lo}.
// Column n = 4 rho + c for realisation rho < nreal.
//   spin 2: c = 0,1: k_l (E + iB) re, im;  c = 2,3: k_l (-1)^(l+m) (E - iB) re, im
//   spin 0: c = 0,1: k_l a re, im;         c = 2,3: k_l (-1)^(l+m) a re, im
struct TcAlm {
  const double *a[2];  // spin 0 field, or E (spin 2)
  const double *b[2];  // B (spin 2), may be NULL
};

__global__ void tcprep_kernel(int lmax, int s, int nreal, TcAlm alm, const long long *__restrict__ blkofs,
                              const float2 *__restrict__ tab, float4 *__restrict__ out) {
  const int m = blockIdx.y;
  const int as = s < 0 ? -s : s;
  const int l0 = m > as ? m : as;
  const int nblk = (lmax >= l0) ? (lmax - l0 + 8) / 8 : 0;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;  // (block, lane)
  if (e >= nblk * 32) return;
  const int blk = e >> 5, lane = e & 31;
  const int g = lane >> 2, t = lane & 3;
  const int rho = g >> 2, c = g & 3;
  float v[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int l = l0 + 8 * blk + t + 4 * h;
    double val = 0.0;
    if (l <= lmax && rho < nreal) {
      const long long idx = (long long)m * (2 * lmax + 1 - m) / 2 + l;
      const double k = (double)tab[idx].x;
      const double sg = ((l + m) & 1) ? -1.0 : 1.0;
      const double *A = alm.a[rho], *Bm = alm.b[rho];
      const double ar = A[2 * idx], ai = (m > 0) ? A[2 * idx + 1] : 0.0;
      if (s == 0) {
        const double re = ar * k, im = ai * k;
        val = (c == 0) ? re : (c == 1) ? im : (c == 2) ? sg * re : sg * im;
      } else {
        const double br = Bm ? Bm[2 * idx] : 0.0, bi = (Bm && m > 0) ? Bm[2 * idx + 1] : 0.0;
        val = (c == 0) ? (ar - bi) * k : (c == 1) ? (ai + br) * k : (c == 2) ? sg * k * (ar + bi) : sg * k * (ai - br);
      }
    }
    v[h] = (float)val;
  }
  float4 r;
  const uint32_t h0 = to_tf32(v[0]), h1 = to_tf32(v[1]);
  r.x = __uint_as_float(h0);
  r.y = __uint_as_float(h1);
  r.z = __uint_as_float(to_tf32(v[0] - __uint_as_float(h0)));
  r.w = __uint_as_float(to_tf32(v[1] - __uint_as_float(h1)));
  out[(blkofs[m] + blk) * 32 + lane] = r;
}

// ---------------------------------------------------------------------------
// shared pieces of the recurrence (same mathematics as legendre.cu)

__host__ __device__ __forceinline__ constexpr int binom_tc(int n, int k) {
  int r = 1;
  for (int t = 1; t <= k; ++t) r = r * (n - k + t) / t;
  return r;
}

template <int NDER>
__device__ __forceinline__ void seed_f32(const RingTable &rt, int r, double E, double a, double b, double sign,
                                         double invL, float (&cur)[NDER + 1], int &sc) {
  typedef RealTraits<float> RT;
  int s0 = (int)ceil((E - RT::H) / (double)RT::SB);
  if (s0 > 0) s0 = 0;
  sc = s0;
  const double mant = sign * exp2(E - (double)RT::SB * s0);
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
    for (int i = 0; i <= j; ++i) acc += (double)binom_tc(j, i) * g[i + 1] * B[j - i];
    B[j + 1] = acc;
  }
  double p = 1.0;
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    cur[j] = (float)(mant * B[j] * p);
    p *= invL;
  }
}

template <int NDER>
__device__ __forceinline__ void leib_f32(double x, double st, double invL, float (&e)[NDER + 1][NDER + 1]) {
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
    for (int i = 0; i <= NDER; ++i) e[j][i] = (i >= 1 && i <= j) ? (float)(binom_tc(j, i) * dc[i]) : 0.0f;
}

template <int NDER>
__device__ __forceinline__ void step_f32(float (&old)[NDER + 1], const float (&cur)[NDER + 1],
                                         const float (&e)[NDER + 1][NDER + 1], float X, float A) {
#pragma unroll
  for (int j = NDER; j >= 0; --j) {
    float acc = X * cur[j];
#pragma unroll
    for (int i = 1; i <= j; ++i) acc = fmaf(e[j][i], cur[j - i], acc);
    old[j] = fmaf(A, acc, -old[j]);
  }
}

template <int NDER>
__device__ __forceinline__ void rescale_f32(float (&a)[NDER + 1], float (&b)[NDER + 1], float lead, int &sc) {
  typedef RealTraits<float> RT;
  if (sc < 0 && fabsf(lead) > RT::THR) {
#pragma unroll
    for (int j = 0; j <= NDER; ++j) {
      a[j] *= RT::STEP;
      b[j] *= RT::STEP;
    }
    ++sc;
  }
}

// Store the current 4 buffered steps of every order into the warp's tiles.
// TF32: round to nearest. 3xTF32: hi = the value with its low 13 mantissa bits
// cleared (exactly a TF32 number), lo = value - hi (exact); the tensor core reads
// the top 19 bits of lo, so the pair carries ~21 bits.
__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

template <int NDER, int MODE>
__device__ __forceinline__ void stash4(float *tile_hi, float *tile_lo, int lane, int chunk,
                                       const float (&buf)[NDER + 1][4]) {
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    float4 h, lo;
    const uint32_t off = tile_off(lane, chunk) + (uint32_t)j * 1024u;
    if (MODE == 3) {
      h.x = tf32_trunc(buf[j][0]);
      h.y = tf32_trunc(buf[j][1]);
      h.z = tf32_trunc(buf[j][2]);
      h.w = tf32_trunc(buf[j][3]);
      lo.x = buf[j][0] - h.x;
      lo.y = buf[j][1] - h.y;
      lo.z = buf[j][2] - h.z;
      lo.w = buf[j][3] - h.w;
      *(float4 *)((char *)tile_hi + off) = h;
      *(float4 *)((char *)tile_lo + off) = lo;
    } else {
      h.x = __uint_as_float(to_tf32(buf[j][0]));
      h.y = __uint_as_float(to_tf32(buf[j][1]));
      h.z = __uint_as_float(to_tf32(buf[j][2]));
      h.w = __uint_as_float(to_tf32(buf[j][3]));
      *(float4 *)((char *)tile_hi + off) = h;
    }
  }
}

// Eight recurrence steps of one block: stash the current values (zero while the
// ring's values are below the representable range unless GATED is false, i.e.
// every lane of the warp is already in range) and step forward.
template <int NDER, int MODE, bool GATED, bool SPIN2>
__device__ __forceinline__ void eight_steps(float (&a)[NDER + 1], float (&b)[NDER + 1], int &sc,
                                            const float (&e)[NDER + 1][NDER + 1], float X, const float (&Av)[8],
                                            const float (&Cv)[8], float *tile_hi, float *tile_lo, int lane) {
  float buf[NDER + 1][4];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const bool on = GATED ? (sc == 0) : true;
#pragma unroll
    for (int j = 0; j <= NDER; ++j) buf[j][s & 3] = on ? ((s & 1) ? a[j] : b[j]) : 0.0f;
    if ((s & 3) == 3) stash4<NDER, MODE>(tile_hi, tile_lo, lane, s >> 2, buf);
    const float Xs = SPIN2 ? X + Cv[s] : X;
    if (s & 1) {
      step_f32<NDER>(b, a, e, Xs, Av[s]);
      if (GATED) rescale_f32<NDER>(a, b, b[0], sc);
    } else {
      step_f32<NDER>(a, b, e, Xs, Av[s]);
      if (GATED) rescale_f32<NDER>(a, b, a[0], sc);
    }
  }
}

// Contract the staged [32 x 8] tiles of orders 0..NJ-1 against one B fragment.
template <int NDER, int NJ, int MODE>
__device__ __forceinline__ void contract(const float *tile_hi, const float *tile_lo, int lane, float4 bf,
                                         float (&acc)[NDER + 1][2][4]) {
  const uint32_t bh0 = __float_as_uint(bf.x), bh1 = __float_as_uint(bf.y);
  const uint32_t bl0 = __float_as_uint(bf.z), bl1 = __float_as_uint(bf.w);
  const uint32_t shi = (uint32_t)__cvta_generic_to_shared(tile_hi);
  const uint32_t slo = (uint32_t)__cvta_generic_to_shared(tile_lo);
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    uint32_t a0[4], a1[4];
    load_afrag(shi + (uint32_t)j * 1024u, lane, a0, a1);
    mma_tf32(acc[j][0], a0, bh0, bh1);
    mma_tf32(acc[j][1], a1, bh0, bh1);
    if (MODE == 3) {
      mma_tf32(acc[j][0], a0, bl0, bl1);
      mma_tf32(acc[j][1], a1, bl0, bl1);
      uint32_t c0[4], c1[4];
      load_afrag(slo + (uint32_t)j * 1024u, lane, c0, c1);
      mma_tf32(acc[j][0], c0, bh0, bh1);
      mma_tf32(acc[j][1], c1, bh0, bh1);
    }
  }
}

// Scatter a warp's accumulator fragments to xch[ring][j][col] (8 columns).
template <int NDER>
__device__ __forceinline__ void acc_to_smem(float *xch, int warp, int lane, const float (&acc)[NDER + 1][2][4],
                                            int nj) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    if (j >= nj) break;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = mt * 16 + g + ((i >> 1) << 3);
        const int col = 2 * t + (i & 1);
        xch[((warp * 32 + row) * (NDER + 1) + j) * 8 + col] = acc[j][mt][i];
      }
  }
}

// ---------------------------------------------------------------------------
// kernel bodies: one (m, ring block) unit of work for a 64-thread block

struct TcDesc {
  RingTable rt;
  const double *lnorm0;
  int nside, lmax, mmax, nrings, nreal;
  const long long *blk;  // first block of each m
  const float *step;     // step factors per block
  const float4 *b;       // coefficient fragments (spin 0: the field; spin 2: E, B)
  const float4 *bp;      // spin 0: the lensing potential's fragments (or NULL)
  float2 *d7a, *d7b;     // spin 0: field, potential planes; spin 2: Q, U planes
  long long rstride, rstride_p;
};

// spin 2: block = 2 warps: 32 north rings (rblk * 32 ..) then their mirrors
template <int NDER, int MODE>
__device__ __forceinline__ void tc2_body(const TcDesc &D, int m, int rblk, float *smem) {
  constexpr int NJ = NDER + 1;
  const RingTable &rt = D.rt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rn = rblk * 32 + lane;
  const bool active = rn < 2 * D.nside;
  const bool mirror = warp == 1;
  const int r = active ? (mirror ? D.nrings - 1 - rn : rn) : 0;
  const double invL = 1.0 / (double)(D.lmax + 1);
  float *tile_hi = smem + (warp * 2 + 0) * NJ * 256;
  float *tile_lo = smem + (warp * 2 + 1) * NJ * 256;

  float e[NJ][NJ];
  float a[NJ], b[NJ];
  int sc = -1;
  const int l0 = m > 2 ? m : 2;
  {
    const double x = rt.z[r], st = rt.sint[r];
    leib_f32<NDER>(x, st, invL, e);
    const double lsh = rt.log2_sh[r], lch = rt.log2_ch[r];
    double E, ea, eb;
    if (m >= 2) {
      const double md = (double)m;
      E = D.lnorm0[m] + 0.5 * log2(md * (md - 1.0) / ((md + 1.0) * (md + 2.0))) + (md + 2.0) * lsh +
          (md - 2.0) * lch;
      ea = md + 2.0;
      eb = md - 2.0;
    } else {
      const double c4 = (m == 0) ? 6.0 : 4.0;
      E = log2(sqrt(5.0 / (4.0 * 3.14159265358979323846)) * sqrt(c4)) + (2.0 + m) * lsh + (2.0 - m) * lch;
      ea = 2.0 + m;
      eb = 2.0 - m;
    }
    seed_f32<NDER>(rt, r, E, ea, eb, (m & 1) ? -1.0 : 1.0, invL, b, sc);
    if (!active) sc = -1000000;  // contributes nothing
  }
#pragma unroll
  for (int j = 0; j < NJ; ++j) a[j] = 0.0f;
  const float X = (float)rt.z[r];

  float acc[NJ][2][4];
#pragma unroll
  for (int j = 0; j < NJ; ++j)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[j][mt][i] = 0.0f;

  const int nblk = (D.lmax >= l0) ? (D.lmax - l0 + 8) / 8 : 0;
  const long long b0 = D.blk[m];
  for (int blk = 0; blk < nblk; ++blk) {
    const float4 *stp = (const float4 *)(D.step + (b0 + blk) * 16);
    const float4 A0 = stp[0], A1 = stp[1], C0 = stp[2], C1 = stp[3];
    const float Av[8] = {A0.x, A0.y, A0.z, A0.w, A1.x, A1.y, A1.z, A1.w};
    const float Cv[8] = {C0.x, C0.y, C0.z, C0.w, C1.x, C1.y, C1.z, C1.w};
    const float4 bf = D.b[(b0 + blk) * 32 + lane];
    if (__all_sync(0xffffffffu, sc == 0))
      eight_steps<NDER, MODE, false, true>(a, b, sc, e, X, Av, Cv, tile_hi, tile_lo, lane);
    else
      eight_steps<NDER, MODE, true, true>(a, b, sc, e, X, Av, Cv, tile_hi, tile_lo, lane);
    __syncwarp();
    contract<NDER, NJ, MODE>(tile_hi, tile_lo, lane, bf, acc);
    __syncwarp();
  }
  __syncthreads();
  float *xch = smem;  // [64 rings][NJ][8]
  acc_to_smem<NDER>(xch, warp, lane, acc, NJ);
  __syncthreads();
  if (!active || m > D.mmax) return;
  if (mirror && rn == D.nrings - 1 - rn) return;  // equator: the north thread writes it
  const int me = warp * 32 + lane, partner = (1 - warp) * 32 + lane;
  const size_t ld = (size_t)(D.mmax + 1);
  for (int rho = 0; rho < D.nreal; ++rho) {
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const float s1r = xch[(me * NJ + j) * 8 + 4 * rho], s1i = xch[(me * NJ + j) * 8 + 4 * rho + 1];
      const float s2r = xch[(partner * NJ + j) * 8 + 4 * rho + 2], s2i = xch[(partner * NJ + j) * 8 + 4 * rho + 3];
      const float sg = (j & 1) ? -1.0f : 1.0f;
      const float ar = s1r + sg * s2r, ai = s1i + sg * s2i;
      const float br = s1r - sg * s2r, bi = s1i - sg * s2i;
      const size_t o = (size_t)rho * D.rstride + ((size_t)j * D.nrings + r) * ld + m;
      D.d7a[o] = make_float2(-0.5f * ar, -0.5f * ai);
      D.d7b[o] = make_float2(-0.5f * bi, 0.5f * br);
    }
  }
}

// spin 0: block = 2 warps of north rings incl. the equator (rblk * 64 ..); south
// by parity. With PHI the potential's fragments are contracted for j <= 1 as well.
template <int NDER, int MODE, bool PHI>
__device__ __forceinline__ void tc0_body(const TcDesc &D, int m, int rblk, float *smem, float *xchp) {
  constexpr int NJ = NDER + 1;
  const RingTable &rt = D.rt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = rblk * 64 + threadIdx.x;  // north ring 0 .. 2N-1
  const bool active = r0 < 2 * D.nside;
  const int r = active ? r0 : 0;
  const double invL = 1.0 / (double)(D.lmax + 1);
  float *tile_hi = smem + (warp * 2 + 0) * NJ * 256;
  float *tile_lo = smem + (warp * 2 + 1) * NJ * 256;

  float e[NJ][NJ];
  float a[NJ], b[NJ];
  int sc = -1;
  {
    const double x = rt.z[r], st = rt.sint[r];
    leib_f32<NDER>(x, st, invL, e);
    const double E = D.lnorm0[m] + (double)m * (rt.log2_sh[r] + rt.log2_ch[r]);
    seed_f32<NDER>(rt, r, E, (double)m, (double)m, (m & 1) ? -1.0 : 1.0, invL, b, sc);
    if (!active) sc = -1000000;
  }
#pragma unroll
  for (int j = 0; j < NJ; ++j) a[j] = 0.0f;
  const float X = (float)rt.z[r];

  float acc[NJ][2][4], accp[2][2][4];
#pragma unroll
  for (int j = 0; j < NJ; ++j)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[j][mt][i] = 0.0f;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int i = 0; i < 4; ++i) accp[j][mt][i] = 0.0f;

  const int nblk = (D.lmax - m + 8) / 8;
  const long long b0 = D.blk[m];
  for (int blk = 0; blk < nblk; ++blk) {
    const float4 *stp = (const float4 *)(D.step + (b0 + blk) * 16);
    const float4 A0 = stp[0], A1 = stp[1];
    const float Av[8] = {A0.x, A0.y, A0.z, A0.w, A1.x, A1.y, A1.z, A1.w};
    const float4 bf = D.b[(b0 + blk) * 32 + lane];
    float4 bp;
    if (PHI) bp = D.bp[(b0 + blk) * 32 + lane];
    const float Cv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (__all_sync(0xffffffffu, sc == 0))
      eight_steps<NDER, MODE, false, false>(a, b, sc, e, X, Av, Cv, tile_hi, tile_lo, lane);
    else
      eight_steps<NDER, MODE, true, false>(a, b, sc, e, X, Av, Cv, tile_hi, tile_lo, lane);
    __syncwarp();
    contract<NDER, NJ, MODE>(tile_hi, tile_lo, lane, bf, acc);
    if (PHI) contract<1, 2, MODE>(tile_hi, tile_lo, lane, bp, accp);
    __syncwarp();
  }
  __syncthreads();
  float *xch = smem;
  acc_to_smem<NDER>(xch, warp, lane, acc, NJ);
  if (PHI) acc_to_smem<1>(xchp, warp, lane, accp, 2);
  __syncthreads();
  if (!active || m > D.mmax) return;
  const int me = warp * 32 + lane;
  const int rs = D.nrings - 1 - r;
  const size_t ld = (size_t)(D.mmax + 1);
  for (int rho = 0; rho < D.nreal; ++rho) {
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const float *x = xch + (me * NJ + j) * 8 + 4 * rho;
      const float sg = (j & 1) ? -1.0f : 1.0f;
      const size_t o = (size_t)rho * D.rstride + (size_t)j * D.nrings * ld + m;
      D.d7a[o + (size_t)r * ld] = make_float2(x[0], x[1]);
      if (rs != r) D.d7a[o + (size_t)rs * ld] = make_float2(sg * x[2], sg * x[3]);
    }
    if (PHI) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float *x = xchp + (me * 2 + j) * 8 + 4 * rho;
        const float sg = (j & 1) ? -1.0f : 1.0f;
        const size_t o = (size_t)rho * D.rstride_p + (size_t)j * D.nrings * ld + m;
        D.d7b[o + (size_t)r * ld] = make_float2(x[0], x[1]);
        if (rs != r) D.d7b[o + (size_t)rs * ld] = make_float2(sg * x[2], sg * x[3]);
      }
    }
  }
}

template <int NDER, int MODE>
__global__ void __launch_bounds__(64) legendre_spin2_tc(TcDesc D) {
  __shared__ __align__(128) float smem[2 * 2 * (NDER + 1) * 256];
  tc2_body<NDER, MODE>(D, blockIdx.y, blockIdx.x, smem);
}

template <int NDER, int MODE, bool PHI>
__global__ void __launch_bounds__(64) legendre_spin0_tc(TcDesc D) {
  __shared__ __align__(128) float smem[2 * 2 * (NDER + 1) * 256];
  __shared__ float xchp[PHI ? 64 * 2 * 8 : 1];
  tc0_body<NDER, MODE, PHI>(D, blockIdx.y, blockIdx.x, smem, xchp);
}

// ---------------------------------------------------------------------------
// persistent form: one launch covers the spin-0 and spin-2 work of several
// plans (geometries). Items (descriptor, kind, m, ring block) are pre-sorted by
// cost; blocks take them in order from an atomic counter until none is left.
// kind: 0 spin 0, 1 spin 0 with the potential, 2 spin 2.

template <int NDER, int MODE>
__global__ void __launch_bounds__(64) legendre_tc_persistent(const TcDesc *__restrict__ descs,
                                                             const int4 *__restrict__ items, int nitems,
                                                             int *__restrict__ counter) {
  __shared__ __align__(128) float smem[2 * 2 * (NDER + 1) * 256];
  __shared__ float xchp[64 * 2 * 8];
  __shared__ int cur;
  for (;;) {
    __syncthreads();  // the previous item's shared-memory readers are done
    if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int it = cur;
    if (it >= nitems) return;
    const int4 w = items[it];
    const TcDesc D = descs[w.x & 0xffff];
    const int kind = w.x >> 16;
    if (kind == 2)
      tc2_body<NDER, MODE>(D, w.y, w.z, smem);
    else if (kind == 1)
      tc0_body<NDER, MODE, true>(D, w.y, w.z, smem, xchp);
    else
      tc0_body<NDER, MODE, false>(D, w.y, w.z, smem, xchp);
  }
}

// ---------------------------------------------------------------------------
// launchers

cudaError_t launch_tcstep(const tl_plan *p, int s, const long long *blkofs, const void *tab, float *out,
                          cudaStream_t st) {
  const int maxe = ((p->lmax + 8) / 8) * 8;
  dim3 grid((maxe + 255) / 256, p->lmax + 1);
  tcstep_kernel<<<grid, 256, 0, st>>>(p->lmax, s, blkofs, (const float2 *)tab, out);
  return cudaGetLastError();
}

cudaError_t launch_tcprep(const tl_plan *p, int s, int nreal, const double *const *a, const double *const *b,
                          const long long *blkofs, const void *tab, void *out, cudaStream_t st) {
  TcAlm alm;
  for (int i = 0; i < 2; ++i) {
    alm.a[i] = (i < nreal) ? a[i] : nullptr;
    alm.b[i] = (i < nreal && b) ? b[i] : nullptr;
  }
  const int maxe = ((p->lmax + 8) / 8) * 32;
  dim3 grid((maxe + 255) / 256, p->lmax + 1);
  tcprep_kernel<<<grid, 256, 0, st>>>(p->lmax, s, nreal, alm, blkofs, (const float2 *)tab, (float4 *)out);
  return cudaGetLastError();
}

static TcDesc make_desc(const tl_plan *p, int spin, int nreal, void *d7a, void *d7b, long long rstride,
                        long long rstride_p) {
  TcDesc D;
  D.rt = p->ring;
  D.lnorm0 = p->lnorm0;
  D.nside = p->nside;
  D.lmax = p->lmax;
  D.mmax = p->mmax;
  D.nrings = p->nrings;
  D.nreal = nreal;
  D.blk = spin == 2 ? p->tc_blk2 : p->tc_blk0;
  D.step = spin == 2 ? p->tc_step2 : p->tc_step0;
  D.b = (const float4 *)(spin == 2 ? p->tc_b2 : p->tc_b0);
  D.bp = (const float4 *)p->tc_bp;
  D.d7a = (float2 *)d7a;
  D.d7b = (float2 *)d7b;
  D.rstride = rstride;
  D.rstride_p = rstride_p;
  return D;
}

// Write the descriptor of a plan's spin-0 or spin-2 work (nreal realisations) to dst.
void tc_desc_write(const tl_plan *p, int spin, int nreal, void *dst) {
  const TcDesc d = spin == 2 ? make_desc(p, 2, nreal, p->d7_Q, p->d7_U, p->d7_rstride, 0)
                             : make_desc(p, 0, nreal, p->d7_T, p->d7_P, p->d7_rstride, p->d7p_rstride);
  memcpy(dst, &d, sizeof d);
}

template <int NDER, int MODE>
static cudaError_t tc2(const tl_plan *p, int nreal, void *dq, void *du, long long rstride, cudaStream_t s) {
  dim3 grid((2 * p->nside + 31) / 32, p->mmax + 1);
  legendre_spin2_tc<NDER, MODE><<<grid, 64, 0, s>>>(make_desc(p, 2, nreal, dq, du, rstride, 0));
  return cudaGetLastError();
}

template <int NDER, int MODE, bool PHI>
static cudaError_t tc0(const tl_plan *p, int nreal, void *d7, void *d7p, long long rstride, long long rstride_p,
                       cudaStream_t s) {
  dim3 grid((2 * p->nside + 63) / 64, p->mmax + 1);
  legendre_spin0_tc<NDER, MODE, PHI><<<grid, 64, 0, s>>>(make_desc(p, 0, nreal, d7, d7p, rstride, rstride_p));
  return cudaGetLastError();
}

template <int NDER, int MODE>
static cudaError_t tcp(const void *descs, const void *items, int nitems, int *counter, int grid, cudaStream_t s) {
  legendre_tc_persistent<NDER, MODE><<<grid, 64, 0, s>>>((const TcDesc *)descs, (const int4 *)items, nitems, counter);
  return cudaGetLastError();
}

cudaError_t launch_legendre_tc_persistent(int nder, int precision, const void *descs, const void *items, int nitems,
                                          int *counter, int grid, cudaStream_t s) {
  const bool x3 = precision == TL_MIXED_TF32x3;
  switch (nder) {
#define CASE(n) \
  case n: return x3 ? tcp<n, 3>(descs, items, nitems, counter, grid, s) : tcp<n, 1>(descs, items, nitems, counter, grid, s);
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

size_t tc_desc_bytes() { return sizeof(TcDesc); }

#define TL_TC_ORDERS(X) X(1) X(2) X(3) X(4) X(5) X(6)

cudaError_t launch_legendre_spin2_tc(const tl_plan *p, int nder, int nreal, void *dq, void *du, long long rstride,
                                     cudaStream_t s) {
  const bool x3 = p->precision == TL_MIXED_TF32x3;
  switch (nder) {
#define CASE(n) \
  case n: return x3 ? tc2<n, 3>(p, nreal, dq, du, rstride, s) : tc2<n, 1>(p, nreal, dq, du, rstride, s);
    TL_TC_ORDERS(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_legendre_spin0_tc(const tl_plan *p, int nder, int nreal, bool phi, void *d7, void *d7p,
                                     long long rstride, long long rstride_p, cudaStream_t s) {
  const bool x3 = p->precision == TL_MIXED_TF32x3;
  switch (nder) {
#define CASE(n)                                                                                   \
  case n:                                                                                         \
    if (phi)                                                                                      \
      return x3 ? tc0<n, 3, true>(p, nreal, d7, d7p, rstride, rstride_p, s)                       \
                : tc0<n, 1, true>(p, nreal, d7, d7p, rstride, rstride_p, s);                      \
    return x3 ? tc0<n, 3, false>(p, nreal, d7, d7p, rstride, rstride_p, s)                        \
              : tc0<n, 1, false>(p, nreal, d7, d7p, rstride, rstride_p, s);
    TL_TC_ORDERS(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

}  // namespace tl
