// Legendre stage with the contraction on the 5th-generation tensor cores
// (tcgen05, operands and accumulators in tensor memory) (Naess & Louis 2013,
// Sec. II.B: the derivative maps of Eq. 4).
//
// The recurrence runs exactly as in legendre.cu: one thread per ring, FP32 values
// with FP64 seeds and exponent scaling, normalised step mu_{l+1} = A X mu_l - mu_{l-1},
// theta-derivatives by Leibniz's rule. A CTA holds 128 rings (spin 2: 64 north
// rings and their mirrors; spin 0: 128 north rings, south by parity) in four
// compute warps, plus one warp that issues the tensor-core work; where tensor
// memory allows, four more compute warps run the second half of each unit's l
// range on the same rings (see run_blocks). Every 8 values of l the compute warps
// write the [128 rings x 8 l] tile of mu^(j) of every derivative order j into
// tensor memory (ring slot t in lane t, the tile's row t), and the issuing warp runs
//     D^(j)[128 x NC] += Mu^(j)[128 x 8] . C[8 x NC]       (tcgen05.mma, kind::tf32)
// with Mu^(j) read from tensor memory and the coefficient tile C from shared
// memory. The NC columns (64, or 32 at the highest order) hold the coefficient
// sets of up to NC/4 realisations that share the basis (4 reals each):
//   spin 2: k_l (E + iB), k_l (-1)^(l+m) (E - iB);   spin 0: k_l a, k_l (-1)^(l+m) a.
// TF32 keeps 10 mantissa bits of each operand; the 3xTF32 form splits both into
// hi + lo and accumulates hi.hi + hi.lo + lo.hi (errors near FP32). The BF16x3
// form splits both into BF16 hi + lo (8 significant bits each) and runs two
// kind::f16 MMAs of K = 16 per order and block: the basis tile is [hi | lo] of
// the block's 8 values of l along K, and the coefficient tiles are [hi ; hi] and
// [lo ; lo], so the two products give hi.hi + lo.hi and hi.lo + lo.lo.
//
// Why 64 columns and the basis in tensor memory: measured on GB300, one CTA's
// chain of these small MMAs advances at ~50 cycles per instruction whatever N is
// up to 128, so the MMA side of a block costs the same for 64 columns as for 32
// and the columns per tile set the realisations served per recurrence. The
// accumulators of 16 realisations (5 orders x 64 columns) and the basis tiles
// (2 x 80 columns for 3xTF32; 2 halves x 2 x 40 for BF16x3) then fill the 512
// columns of tensor memory (one CTA per SM).
//
// Pipeline: the basis tiles (tensor memory) and the coefficient tiles (shared
// memory) are double-buffered where the columns allow. For block g the compute
// warps run 8 steps in registers (step factors and coefficient tiles prefetched
// one block ahead), wait until the MMAs of the block that last used the buffer
// have completed (mbarrier "done" of the buffer, signalled by tcgen05.commit),
// store the basis tiles (tcgen05.st) and the coefficient tile, and arrive on the
// buffer's "full" barrier (one arrival per warp). The issuing warp waits for the
// four arrivals, issues the block's MMAs and commits them to the buffer's "done",
// so the tensor core works on one buffer while the other is being filled. With two
// halves each has its own buffers and barriers, and the issuing warp alternates
// between them block by block.
//
// The coefficient tile uses the K-major shared-memory layout without swizzle:
// 8-row x 16-byte core matrices, 128 bytes apart along K and 256 bytes apart along
// the rows. Every wait is bounded; on time-out the kernel records an error flag,
// waits (bounded) for its own MMAs, frees its tensor memory and returns.
#include <math.h>
#include <string.h>

#include "legendre.cuh"

namespace tl {

constexpr int kMaxReal = TL_MAX_BATCH;  // realisations per launch at most (64 columns)
constexpr int kComputeThreads = 128;  // compute threads per half (umma_threads: the CTA's)
// spin-2 epilogue exchange: [128 rings][9] float2 (8 used; the odd row length puts the
// 32 rows a warp writes or reads at once on distinct bank pairs)
constexpr int kXchRow = 9;
constexpr uint32_t kXchBytes = 128 * kXchRow * 8;

// accumulator columns per order for NDER theta-derivatives: 64 (16 realisations)
// up to NDER = 5, 32 (8) at NDER = 6, where 64 would not fit tensor memory
__host__ __device__ constexpr int tc_cols(int nder) { return nder <= 5 ? 64 : 32; }
// coefficient tile of NC columns in shared memory: hi [NC x 8] then lo, TF32
// (BF16x3: [hi ; hi] then [lo ; lo], NC x 16 BF16 each); the same bytes either way
__host__ __device__ constexpr uint32_t btile_bytes(int nc) { return (uint32_t)nc * 64u; }

// contraction forms of the tensor-core kernels (template parameter MODE)
constexpr int kModeTf32 = 1, kModeTf32x3 = 3, kModeBf16x3 = 4;
inline int tc_mode(int precision) {
  return precision == TL_MIXED_TF32x3 ? kModeTf32x3 : precision == TL_MIXED_BF16x3 ? kModeBf16x3 : kModeTf32;
}

// ---------------------------------------------------------------------------
// tcgen05 building blocks

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, no-swizzle tile: byte offset of (row, k) for 4-byte elements
__host__ __device__ __forceinline__ uint32_t can_off(int row, int k) {
  return (uint32_t)((row >> 3) * 256 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// shared-memory matrix descriptor: start, leading (K) byte offset 128, stride (row group) 256
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)(256u >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of tcgen05
  return d;
}

// instruction descriptor: D f32, A and B tf32 (BF16: bf16), both K-major, M = 128, N = NC
template <int NC, bool BF16 = false> struct Idesc {
  static constexpr uint32_t ab = BF16 ? 1u : 2u;
  static constexpr uint32_t value =
      (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(NC >> 3) << 17) | ((128u >> 4) << 24);
};

// D (tensor memory) += A (tensor memory: row i in lane i, K along 8 columns) . B (shared memory)
template <int NC>
__device__ __forceinline__ void umma_tf32_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t db, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(db), "n"(Idesc<NC>::value), "r"(accumulate));
}

// the same with A and B in BF16, K = 16 (A: two values per tensor-memory column,
// the lower k in the low half)
template <int NC>
__device__ __forceinline__ void umma_bf16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t db, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(db), "n"(Idesc<NC, true>::value), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

// bounded wait for the completion of the mbarrier phase with the given parity: at
// most `polls` tries; gives up early when another thread of the CTA has recorded a
// failure in *abort
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int polls,
                                          const volatile int *abort = nullptr) {
  for (int it = 0; it < polls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (abort && (it & 255) == 255 && *abort) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// 32 consecutive columns of the calling thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 or 16 consecutive columns of the calling thread's lane
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[16]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
               "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
      : "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// 3xTF32 split of the basis values: hi = the value with its low 13 mantissa bits
// cleared (exactly a TF32 number), lo = value - hi (exact; the tensor core reads
// its top 19 bits), so the pair carries ~21 bits
__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }
// two floats rounded to BF16 (nearest even) in one word: x0 in the low half
__device__ __forceinline__ uint32_t bf16x2(float x0, float x1) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(x1), "f"(x0));
  return r;
}
// BF16x3 split of a pair: hi = the BF16 roundings, lo = the BF16 roundings of the
// (exact) remainders
__device__ __forceinline__ void bf16_split2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
  hi = bf16x2(x0, x1);
  lo = bf16x2(x0 - __uint_as_float(hi << 16), x1 - __uint_as_float(hi & 0xffff0000u));
}

// Halves of the l range a unit is split into (two sets of compute warps on the
// same rings, see run_blocks): 2 where both halves' basis tiles fit the 512
// columns double-buffered, else 1.
__host__ __device__ constexpr int tc_halves(int nj, int mode, int nc) {
  return nj * nc + 4 * nj * (mode == kModeTf32x3 ? 16 : 8) <= 512 ? 2 : 1;
}

// Tensor-memory map of a CTA: accumulators D^(j) at columns NC j (j < NJ), then
// NH x NB sets of basis tiles: Mu^(j) of half h, buffer i at A0 + (h NB + i) ASET +
// AW j (hi in 8 columns, then lo for 3xTF32; BF16x3: hi pairs in 4 columns, lo
// pairs in 4). Two buffers per half where they fit the 512 columns, else one. The
// allocation is the next power of two; `ctas` is how many CTAs of that size fit the
// SM (at most 4).
template <int NJ, int MODE, int NC, int NH = 1> struct TmemMap {
  static constexpr int AW = MODE == kModeTf32x3 ? 16 : 8;
  static constexpr int A0 = NJ * NC;
  static constexpr int ASET = NJ * AW;
  static constexpr int NB = A0 + NH * 2 * ASET <= 512 ? 2 : 1;
  static constexpr int need = A0 + NH * NB * ASET;
  static constexpr int cols = need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;
  static constexpr int ctas = 512 / cols > 4 ? 4 : 512 / cols;
  static_assert(need <= 512, "tensor memory");
};

// Descriptor of one plan's Legendre work for one coefficient set: a spin-0 field
// (the temperature, or the lensing potential at NDER = 1) or the spin-2 pair (E, B).
struct TcDesc {
  RingTable rt;
  const double *lnorm0;
  int nside, lmax, mmax, nrings, nreal;
  const long long *blk;          // first 8-l block of each m
  const float *step;             // per block: A_{l+1} x 8, then Q x 8 (spin 2: Qn, Qs), see step_stride
  const unsigned char *b;        // per block: coefficient tile hi [NC x 8] then lo
  float2 *d7a, *d7b;             // spin 0: the field's planes; spin 2: Q, U planes
  long long rstride;             // T2 elements between realisations' planes
  int prows;                     // rows of a plane (the rings rounded up to 4: interleaved layout)
  int *err;                      // set to 1 when a wait times out
  // start table (plan-time, tcstart_kernel): per unit m * nrblk + rblk the first
  // 8-l block in which one of its rings contributes, and every ring's recurrence
  // state at the start of that block: [unit][2 NJ + 1][128] (a, b, scale)
  const int *bstart;
  const float *state;
  // the same state at the first block of the unit's second half (see run_blocks),
  // or NULL (no split)
  const float *state_mid;
  int nrblk;
  int polls;  // polls of every mbarrier wait before it gives up (bounded waits)
  int stall;  // self-test: the compute warps withhold their arrivals, so waits run out
};

// Per-CTA tcgen05 state (identical in every thread). Each half h of the compute
// warps has four mbarriers, adjacent 8-byte words from bars + 32 h: done[0],
// done[1] (MMAs of the buffer's last block completed; one arrival, the commit),
// full[0], full[1] (the block's tiles written; one arrival per compute warp of the
// half). Their addresses are formed arithmetically: a runtime-indexed array member
// would put the struct in local memory.
struct UmmaCta {
  uint32_t tmem;        // tensor-memory base (lane 0, first column)
  uint32_t bars;        // shared address of half 0's done[0]
  uint32_t count;       // blocks so far, first half
  uint32_t count1;      // blocks so far, second half
  volatile int *abort;  // shared: set by a thread whose wait timed out
  bool failed;
};
__device__ __forceinline__ uint32_t bar_done(const UmmaCta &U, uint32_t i, uint32_t h = 0) {
  return U.bars + 32u * h + 8u * i;
}
__device__ __forceinline__ uint32_t bar_full(const UmmaCta &U, uint32_t i, uint32_t h = 0) {
  return U.bars + 32u * h + 16u + 8u * i;
}
// threads of a CTA with NH halves: 4 compute warps, the issuing warp, 4 more compute warps
__host__ __device__ constexpr int umma_threads(int nh) { return nh == 2 ? 288 : 160; }
// Block g uses buffer g % NB; it is that buffer's (g / NB)-th use, i.e. phase
// g / NB of both of its barriers.
template <int NB> __device__ __forceinline__ uint32_t buf_of(uint32_t g) { return NB == 2 ? (g & 1u) : 0u; }
template <int NB> __device__ __forceinline__ uint32_t phase_of(uint32_t g) { return (NB == 2 ? (g >> 1) : g) & 1u; }

// ---------------------------------------------------------------------------
// recurrence steps with the basis values buffered for the tiles

// Four steps of the difference form (SG = sign cos th of the thread's ring), the
// basis value of each l saved for the tiles before its step: state (b, a) =
// (mu_l, d_l), step factors A and Q of the block's 8 values of l.
template <int S0, int NDER, bool GATED, int SG>
__device__ __forceinline__ void four_steps(float (&a)[NDER + 1], float (&b)[NDER + 1], int &sc,
                                           const Leib<float, NDER> &LC, float w, const float (&Av)[8],
                                           const float (&Qv)[8], float (&buf)[NDER + 1][4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int s = S0 + q;
    const bool on = GATED ? (sc == 0) : true;
#pragma unroll
    for (int j = 0; j <= NDER; ++j) buf[j][q] = on ? b[j] : 0.0f;
    step_diff<float, NDER, SG>(b, a, LC, w, Av[s], Qv[s]);
    if (GATED) rescale<float, NDER>(a, b, b[0], sc);
  }
}

template <int S0, int NDER, int SG>
__device__ __forceinline__ void steps_gated(float (&a)[NDER + 1], float (&b)[NDER + 1], int &sc,
                                            const Leib<float, NDER> &LC, float w, const float (&Av)[8],
                                            const float (&Qv)[8], float (&buf)[NDER + 1][4]) {
  if (__all_sync(0xffffffffu, sc == 0))
    four_steps<S0, NDER, false, SG>(a, b, sc, LC, w, Av, Qv, buf);
  else
    four_steps<S0, NDER, true, SG>(a, b, sc, LC, w, Av, Qv, buf);
}

// The 8 steps of one block; spin 2's mirror rings (cos th < 0) are whole warps
// (threads 64-127 of a half), so the branch is warp-uniform.
template <int NDER, bool SPIN2>
__device__ __forceinline__ void block_steps(bool mirror, float (&a)[NDER + 1], float (&b)[NDER + 1], int &sc,
                                            const Leib<float, NDER> &LC, float w, const float (&Av)[8],
                                            const float (&Qv)[8], float (&buf0)[NDER + 1][4],
                                            float (&buf1)[NDER + 1][4]) {
  if (SPIN2 && mirror) {
    steps_gated<0, NDER, -1>(a, b, sc, LC, w, Av, Qv, buf0);
    steps_gated<4, NDER, -1>(a, b, sc, LC, w, Av, Qv, buf1);
  } else {
    steps_gated<0, NDER, 1>(a, b, sc, LC, w, Av, Qv, buf0);
    steps_gated<4, NDER, 1>(a, b, sc, LC, w, Av, Qv, buf1);
  }
}

// step table per 8-l block: A_{l+1} x 8, then Q x 8 (spin 0: A - 2; spin 2: Qn x 8
// for rings with cos th >= 0, then Qs x 8 for the mirror rings)
__host__ __device__ constexpr int step_stride(bool spin2) { return spin2 ? 24 : 16; }

// the block's basis values of every order into the calling thread's lane: hi (and
// lo for 3xTF32) of l = l0 + 8 blk + 0..7, at column a0 + AW j; BF16x3: the hi
// pairs (l, l + 1) in 4 columns, then the lo pairs
template <int NDER, int MODE>
__device__ __forceinline__ void store_tiles(uint32_t a0, const float (&buf0)[NDER + 1][4],
                                            const float (&buf1)[NDER + 1][4]) {
  constexpr int AW = MODE == kModeTf32x3 ? 16 : 8;
#pragma unroll
  for (int j = 0; j <= NDER; ++j) {
    float v[16];
    if (MODE == kModeBf16x3) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float x0 = q < 2 ? buf0[j][2 * q] : buf1[j][2 * q - 4];
        const float x1 = q < 2 ? buf0[j][2 * q + 1] : buf1[j][2 * q - 3];
        uint32_t hi, lo;
        bf16_split2(x0, x1, hi, lo);
        v[q] = __uint_as_float(hi);
        v[4 + q] = __uint_as_float(lo);
      }
      tmem_st8(a0 + (uint32_t)(AW * j), v);
      continue;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float x = k < 4 ? buf0[j][k] : buf1[j][k - 4];
      if (MODE == kModeTf32x3) {
        v[k] = tf32_trunc(x);
        v[8 + k] = x - v[k];
      } else {
        v[k] = __uint_as_float(to_tf32(x));
      }
    }
    if (MODE == kModeTf32x3)
      tmem_st16(a0 + (uint32_t)(AW * j), v);
    else
      tmem_st8(a0 + (uint32_t)(AW * j), v);
  }
}

// D^(j) += Mu^(j) . C for j < NJ (and the lo terms for 3xTF32 and BF16x3), basis
// tiles at column aset, coefficient tile at descriptor dB (its lo half btile/2 bytes on)
template <int NJ, int MODE, int NC>
__device__ __forceinline__ void issue_block(uint32_t tmem, uint32_t aset, uint64_t dB, bool first) {
  typedef TmemMap<NJ, MODE, NC> TM;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const uint32_t d = tmem + (uint32_t)(NC * j), a = tmem + aset + (uint32_t)(TM::AW * j);
    if (MODE == kModeBf16x3) {
      umma_bf16_ts<NC>(d, a, dB, first ? 0u : 1u);                     // [hi | lo] . [hi ; hi]
      umma_bf16_ts<NC>(d, a, dB + ((btile_bytes(NC) / 2) >> 4), 1u);  // [hi | lo] . [lo ; lo]
      continue;
    }
    umma_tf32_ts<NC>(d, a, dB, first ? 0u : 1u);
    if (MODE == kModeTf32x3) {
      umma_tf32_ts<NC>(d, a, dB + ((btile_bytes(NC) / 2) >> 4), 1u);  // hi . lo
      umma_tf32_ts<NC>(d, a + 8u, dB, 1u);                             // lo . hi
    }
  }
}

__device__ __forceinline__ int unit_l0(int m, bool spin2) { return spin2 ? (m > 2 ? m : 2) : m; }

// ring of compute thread tid in ring block rblk (spin 2: 64 north rings, then
// their mirrors; spin 0: 128 north rings); inactive threads past the equator
// take ring 0 and contribute nothing
template <bool SPIN2>
__device__ __forceinline__ int unit_ring(const TcDesc &D, int rblk, int tid, bool &active) {
  const int rn = SPIN2 ? rblk * 64 + (tid & 63) : rblk * 128 + tid;
  active = rn < 2 * D.nside;
  if (!active) return 0;
  return (SPIN2 && tid >= 64) ? D.nrings - 1 - rn : rn;
}

// recurrence state at l0: mu_{l0} in b, d_{l0} = mu_{l0} in a, scale sc
template <int NDER, bool SPIN2>
__device__ __forceinline__ void unit_seed(const TcDesc &D, int r, int m, bool active, float (&a)[NDER + 1],
                                          float (&b)[NDER + 1], int &sc) {
  const double invL = 1.0 / (double)(D.lmax + 1);
  if (SPIN2)
    (void)seed_spin2<float, NDER>(D.rt, D.lnorm0, r, m, invL, b, sc);
  else
    seed_spin0<float, NDER>(D.rt, D.lnorm0, r, m, invL, b, sc);
  if (!active) sc = -1000000;  // contributes nothing
  rec_init<float, NDER>(a, b);  // difference form: d = mu_{l0}
}

// One (m, ring block) unit: recurrence and tiles (compute warps), MMAs (issuing
// warp). NB: the kernel's buffer count per half (the same for every unit a CTA
// runs, so that the barriers' phases follow one block count). NH = 2 splits the
// unit's blocks between two sets of four compute warps on the same 128 rings: the
// first runs blocks [bs, bmid) from the start-table state, the second [bmid, nblk)
// from the state the recurrence has at bmid (plan-time table state_mid, identical
// arithmetic), and both feed the same accumulators; warps 0-3 form the first set,
// warps 5-8 the second (ring 32 (warp mod 4) + lane: the tensor-memory lanes a warp
// may access). Leaves the accumulators complete in tensor memory (every MMA waited
// for) and returns the number of 8-l blocks run (0: accumulators unset).
template <int NDER, int MODE, int NC, int NB, bool SPIN2, int NH>
__device__ __forceinline__ int run_blocks(const TcDesc &D, int m, int rblk, unsigned char *sm, UmmaCta &U) {
  constexpr int NJ = NDER + 1;
  typedef TmemMap<NJ, MODE, NC, NH> TM;
  static_assert(NB <= TM::NB, "buffers fit");
  constexpr uint32_t BT = btile_bytes(NC);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int l0 = unit_l0(m, SPIN2);
  const int nblk = (D.lmax >= l0) ? (D.lmax - l0 + 8) / 8 : 0;
  const long long b0 = D.blk[m];
  const long long unit = (long long)m * D.nrblk + rblk;
  // blocks before bs contribute nothing for any ring of the unit (start table)
  const int bs = D.bstart ? D.bstart[unit] : 0;
  const int nrun = nblk - bs;
  const bool split = NH == 2 && D.bstart && D.state_mid;
  const int n0 = split ? (nrun + 1) / 2 : nrun, n1 = nrun - n0;
  const uint32_t g00 = U.count, g01 = U.count1;
  bool bad = false;
  if (warp == kComputeThreads / 32) {
    // ---- issuing warp: one lane waits for each block's tiles and issues its MMAs,
    // block k of the first half, then block k of the second
    if (tid == kComputeThreads) {
      const uint64_t dB0 = umma_desc(smem_u32(sm));
      for (int k = 0; k < n0 && !bad; ++k) {
#pragma unroll
        for (int h = 0; h < NH; ++h) {
          if (h == 1 && k >= n1) break;
          const uint32_t g = (h ? g01 : g00) + (uint32_t)k, i = buf_of<NB>(g), ib = (uint32_t)h * NB + i;
          if (!mbar_wait(bar_full(U, i, h), phase_of<NB>(g), D.polls, U.abort)) {
            bad = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          issue_block<NJ, MODE, NC>(U.tmem, (uint32_t)(TM::A0 + TM::ASET * ib), dB0 + ((ib * BT) >> 4),
                                    h == 0 && k == 0);
          umma_commit(bar_done(U, i, h));
        }
      }
    }
    __syncwarp();
  } else {
    // ---- compute warps: one ring per thread (tensor-memory lane t)
    const int h = (NH == 2 && warp > kComputeThreads / 32) ? 1 : 0;
    const int t = h ? (((warp & 3) << 5) | (tid & 31)) : tid;
    const int first = h ? bs + n0 : bs, cnt = h ? n1 : n0;
    const uint32_t g0 = h ? g01 : g00;
    const RingTable &rt = D.rt;
    bool active;
    const int r = unit_ring<SPIN2>(D, rblk, t, active);
    const uint32_t lane = U.tmem + ((uint32_t)((warp & 3) * 32) << 16);
    Leib<float, NDER> LC;
    leibniz_coefs<float, NDER>(rt.z[r], rt.sint[r], 1.0 / (double)(D.lmax + 1), LC);
    float a[NJ], b[NJ];
    int sc;
    if (D.bstart) {
      // the state at block `first`, as the recurrence from l0 leaves it
      const float *st = (h ? D.state_mid : D.state) + unit * (2 * NJ + 1) * kComputeThreads + t;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        a[j] = __ldg(st + j * kComputeThreads);
        b[j] = __ldg(st + (NJ + j) * kComputeThreads);
      }
      sc = __float_as_int(__ldg(st + 2 * NJ * kComputeThreads));
    } else {
      unit_seed<NDER, SPIN2>(D, r, m, active, a, b, sc);
    }
    const float w = (float)rt.omza[r];
    const bool mirror = SPIN2 && t >= 64;
    // the next block's step factors and coefficient tile (BT / 128 bytes per
    // thread), loaded one block ahead
    constexpr int QV = (int)(BT / 16 / kComputeThreads);  // float4 per thread: 1 or 2
    const int qo = mirror ? 4 : 2;  // float4 offset of the thread's Q values
    float4 nA0 = make_float4(0.f, 0.f, 0.f, 0.f), nA1 = nA0, nC0 = nA0, nC1 = nA0, nbq[QV];
#pragma unroll
    for (int q = 0; q < QV; ++q) nbq[q] = nA0;
    auto prefetch = [&](int blk) {
      const float4 *stp = (const float4 *)(D.step + (b0 + blk) * step_stride(SPIN2));
      nA0 = __ldg(stp);
      nA1 = __ldg(stp + 1);
      nC0 = __ldg(stp + qo);
      nC1 = __ldg(stp + qo + 1);
      const float4 *bt = (const float4 *)(D.b + (b0 + blk) * BT);
#pragma unroll
      for (int q = 0; q < QV; ++q) nbq[q] = __ldg(bt + q * kComputeThreads + t);
    };
    if (cnt > 0) prefetch(first);
    for (int k = 0; k < cnt; ++k) {
      const int blk = first + k;
      const uint32_t g = g0 + (uint32_t)k, i = buf_of<NB>(g), ib = (uint32_t)h * NB + i;
      const float Av[8] = {nA0.x, nA0.y, nA0.z, nA0.w, nA1.x, nA1.y, nA1.z, nA1.w};
      const float Cv[8] = {nC0.x, nC0.y, nC0.z, nC0.w, nC1.x, nC1.y, nC1.z, nC1.w};
      float4 bq[QV];
#pragma unroll
      for (int q = 0; q < QV; ++q) bq[q] = nbq[q];
      if (k + 1 < cnt) prefetch(blk + 1);
      float buf0[NJ][4], buf1[NJ][4];
      block_steps<NDER, SPIN2>(mirror, a, b, sc, LC, w, Av, Cv, buf0, buf1);
      // the buffer was last read by the MMAs of this half's block g - NB
      if (g >= (uint32_t)NB && !mbar_wait(bar_done(U, i, h), phase_of<NB>(g - NB), D.polls, U.abort)) {
        bad = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int q = 0; q < QV; ++q) *(float4 *)(sm + ib * BT + (q * kComputeThreads + t) * 16) = bq[q];
      store_tiles<NDER, MODE>(lane + (uint32_t)(TM::A0 + TM::ASET * ib), buf0, buf1);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if ((tid & 31) == 0 && !D.stall) mbar_arrive(bar_full(U, i, h));
    }
  }
  U.count = g00 + (uint32_t)n0;
  U.count1 = g01 + (uint32_t)n1;
  // the last commit of each half covers every MMA issued before it
  if (!bad && n0 > 0 &&
      !mbar_wait(bar_done(U, buf_of<NB>(U.count - 1), 0), phase_of<NB>(U.count - 1), D.polls, U.abort))
    bad = true;
  if (NH == 2 && !bad && n1 > 0 &&
      !mbar_wait(bar_done(U, buf_of<NB>(U.count1 - 1), 1), phase_of<NB>(U.count1 - 1), D.polls, U.abort))
    bad = true;
  if (bad) *U.abort = 1;
  if (__syncthreads_or(bad)) {
    U.failed = true;
    return 0;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return nrun;
}

// Dynamic shared memory of a CTA: two coefficient tile buffers per half, then the
// spin-2 exchange area.
template <int NC, int NH> __host__ __device__ constexpr uint32_t xch_offset() { return 2 * NH * btile_bytes(NC); }

// spin 2: combine each ring's S1 with its mirror's S2 into F^Q, F^U, one order and
// one group of 8 realisations (32 columns) at a time
template <int NDER, int MODE, int NC, int NB, int NH>
__device__ __forceinline__ void u2_unit(const TcDesc &D, int m, int rblk, unsigned char *sm, UmmaCta &U) {
  constexpr int NJ = NDER + 1;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nblk = run_blocks<NDER, MODE, NC, NB, true, NH>(D, m, rblk, sm, U);
  if (U.failed) return;
  const bool compute = tid < kComputeThreads;
  const int rn = rblk * 64 + (tid & 63);
  const bool active = compute && rn < 2 * D.nside;
  const bool mirror = tid >= 64;
  const int r = active ? (mirror ? D.nrings - 1 - rn : rn) : 0;
  const bool writer = active && m <= D.mmax && !(mirror && rn == D.nrings - 1 - rn);  // equator: north thread
  const int partner = tid ^ 64;
  const size_t ld = (size_t)(D.mmax + 1);
  float2 *xch = (float2 *)(sm + xch_offset<NC, NH>());  // [128][kXchRow]: S2 (4 rho + 2, 3) of every ring
#pragma unroll 1
  for (int j = 0; j < NJ; ++j) {
#pragma unroll 1
    for (int h = 0; h < NC / 32; ++h) {
      float v[32];
      if (compute) {
        tmem_ld32(U.tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(NC * j + 32 * h), v);
#pragma unroll
        for (int rho = 0; rho < 8; ++rho) {
          xch[tid * kXchRow + rho] = nblk ? make_float2(v[4 * rho + 2], v[4 * rho + 3]) : make_float2(0.f, 0.f);
        }
      }
      __syncthreads();
      if (writer) {
        const float sg = (j & 1) ? -1.0f : 1.0f;
#pragma unroll
        for (int rho = 0; rho < 8; ++rho) {
          if (8 * h + rho >= D.nreal) break;
          const float s1r = nblk ? v[4 * rho] : 0.f, s1i = nblk ? v[4 * rho + 1] : 0.f;
          const float2 s2 = xch[partner * kXchRow + rho];
          const float s2r = s2.x, s2i = s2.y;
          const float ar = s1r + sg * s2r, ai = s1i + sg * s2i;
          const float br = s1r - sg * s2r, bi = s1i - sg * s2i;
          const size_t o = (size_t)(8 * h + rho) * D.rstride + (size_t)j * D.prows * ld + d7_il(r, m, ld);
          D.d7a[o] = make_float2(-0.5f * ar, -0.5f * ai);
          D.d7b[o] = make_float2(-0.5f * bi, 0.5f * br);
        }
      }
      __syncthreads();  // xch is rewritten next
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// spin 0: north ring r and its mirror by parity
template <int NDER, int MODE, int NC, int NB, int NH>
__device__ __forceinline__ void u0_unit(const TcDesc &D, int m, int rblk, unsigned char *sm, UmmaCta &U) {
  constexpr int NJ = NDER + 1;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nblk = run_blocks<NDER, MODE, NC, NB, false, NH>(D, m, rblk, sm, U);
  if (U.failed) return;
  if (tid < kComputeThreads) {
    const int rn = rblk * 128 + tid;
    const bool active = rn < 2 * D.nside && m <= D.mmax;
    const int r = active ? rn : 0;
    const int rs = D.nrings - 1 - r;
    const size_t ld = (size_t)(D.mmax + 1);
    const uint32_t lane_base = U.tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int j = 0; j < NJ; ++j) {
      const float sg = (j & 1) ? -1.0f : 1.0f;
#pragma unroll 1
      for (int h = 0; h < NC / 32; ++h) {
        float v[32];
        tmem_ld32(lane_base + (uint32_t)(NC * j + 32 * h), v);
        if (!active) continue;
        if (nblk == 0) {  // nothing contributed: the accumulators were not written
#pragma unroll
          for (int c = 0; c < 32; ++c) v[c] = 0.f;
        }
#pragma unroll
        for (int rho = 0; rho < 8; ++rho) {
          if (8 * h + rho >= D.nreal) break;
          const size_t o = (size_t)(8 * h + rho) * D.rstride + (size_t)j * D.prows * ld;
          D.d7a[o + d7_il(r, m, ld)] = make_float2(v[4 * rho], v[4 * rho + 1]);
          if (rs != r) D.d7a[o + d7_il(rs, m, ld)] = make_float2(sg * v[4 * rho + 2], sg * v[4 * rho + 3]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
}

// CTA set-up and tear-down of the barriers (4 per half, `bars` holds 8) and the
// tensor memory
template <int NCOLS, int NH>
__device__ __forceinline__ void umma_open(UmmaCta &U, uint64_t *bars, uint32_t *tbase, int *abort) {
  if (threadIdx.x == 0) {
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[4 * h])));      // done[0]: the commit
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[4 * h + 1])));  // done[1]
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&bars[4 * h + 2])));  // full[0]: 4 warps
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&bars[4 * h + 3])));  // full[1]
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    *abort = 0;
  }
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tbase)),
                 "n"(NCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  U.tmem = *tbase;
  U.bars = smem_u32(&bars[0]);
  U.count = 0;
  U.count1 = 0;
  U.abort = abort;
  U.failed = false;
}

// NB: the buffers of the kernel's main unit type; the last block's commit of each
// half covers every MMA issued before it.
template <int NCOLS, int NB, int NH>
__device__ __forceinline__ void umma_close(const TcDesc &D, UmmaCta &U) {
  if (U.failed && threadIdx.x == 0) {
    atomicExch(D.err, 1);
    // own MMAs in flight (bounded)
    if (U.count > 0) (void)mbar_wait(bar_done(U, buf_of<NB>(U.count - 1), 0), phase_of<NB>(U.count - 1), D.polls);
    if (NH == 2 && U.count1 > 0)
      (void)mbar_wait(bar_done(U, buf_of<NB>(U.count1 - 1), 1), phase_of<NB>(U.count1 - 1), D.polls);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(U.tmem), "n"(NCOLS));
}

template <int NDER, int MODE>
struct Tc {
  static constexpr int NC = tc_cols(NDER);
  static constexpr int NH = tc_halves(NDER + 1, MODE, NC);
  typedef TmemMap<NDER + 1, MODE, NC, NH> TM;
};

template <int NDER, int MODE>
__global__ void __launch_bounds__(umma_threads(Tc<NDER, MODE>::NH), (Tc<NDER, MODE>::TM::ctas))
    legendre_spin2_umma(TcDesc D) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bars[8];
  __shared__ uint32_t tbase;
  __shared__ int abort_flag;
  typedef Tc<NDER, MODE> C;
  typedef typename C::TM TM;
  UmmaCta U;
  umma_open<TM::cols, C::NH>(U, bars, &tbase, &abort_flag);
  u2_unit<NDER, MODE, C::NC, TM::NB, C::NH>(D, blockIdx.y, blockIdx.x, sm, U);
  umma_close<TM::cols, TM::NB, C::NH>(D, U);
}

// spin 0 at NDER with the column count CNC (the potential runs at NDER = 1 with the
// columns of the plan's order)
template <int NDER, int MODE, int CNC>
struct Tc0 {
  static constexpr int NH = tc_halves(NDER + 1, MODE, CNC);
  typedef TmemMap<NDER + 1, MODE, CNC, NH> TM;
};
template <int NDER, int MODE, int CNC>
__global__ void __launch_bounds__(umma_threads(Tc0<NDER, MODE, CNC>::NH), (Tc0<NDER, MODE, CNC>::TM::ctas))
    legendre_spin0_umma(TcDesc D) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bars[8];
  __shared__ uint32_t tbase;
  __shared__ int abort_flag;
  typedef Tc0<NDER, MODE, CNC> C;
  typedef typename C::TM TM;
  UmmaCta U;
  umma_open<TM::cols, C::NH>(U, bars, &tbase, &abort_flag);
  u0_unit<NDER, MODE, CNC, TM::NB, C::NH>(D, blockIdx.y, blockIdx.x, sm, U);
  umma_close<TM::cols, TM::NB, C::NH>(D, U);
}

// Persistent form: one launch covers the Legendre work of several plans. Items
// (descriptor, kind, m, ring block) are pre-sorted by cost; each CTA takes them in
// order from an atomic counter until none is left (no waits between CTAs). Kinds:
// 0 a spin-0 field at NDER, 1 the lensing potential (spin 0, NDER = 1), 2 spin 2.
// Every kind's tensor-memory map fits the allocation of NDER's, with NDER's halves.
template <int NDER, int MODE>
__global__ void __launch_bounds__(umma_threads(Tc<NDER, MODE>::NH), (Tc<NDER, MODE>::TM::ctas))
    legendre_umma_persistent(const TcDesc *__restrict__ descs, const int4 *__restrict__ items, int nitems,
                             int *__restrict__ counter) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bars[8];
  __shared__ uint32_t tbase;
  __shared__ int abort_flag;
  __shared__ int cur;
  typedef Tc<NDER, MODE> C;
  constexpr int NC = C::NC, NH = C::NH;
  typedef typename C::TM TM;
  typedef TmemMap<2, MODE, NC, NH> TM1;
  static_assert(TM1::A0 + NH * TM::NB * TM1::ASET <= TM::cols, "potential units fit the allocation");
  UmmaCta U;
  umma_open<TM::cols, NH>(U, bars, &tbase, &abort_flag);
  TcDesc D = descs[0];
  for (;;) {
    __syncthreads();  // the previous item's readers of `cur` are done
    if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int it = cur;
    if (it >= nitems) break;
    const int4 w = items[it];
    D = descs[w.x & 0xffff];
    const int kind = w.x >> 16;
    if (kind == 2)
      u2_unit<NDER, MODE, NC, TM::NB, NH>(D, w.y, w.z, sm, U);
    else if (kind == 1)
      u0_unit<1, MODE, NC, TM::NB, NH>(D, w.y, w.z, sm, U);
    else
      u0_unit<NDER, MODE, NC, TM::NB, NH>(D, w.y, w.z, sm, U);
    if (U.failed) break;  // uniform: set after a block-wide vote
  }
  umma_close<TM::cols, TM::NB, NH>(D, U);
}

// Plan-time start table (see TcDesc): one CTA of 128 threads per unit runs the
// recurrence block by block, without the contraction, until one of its rings has
// reached scale 0 (a basis value that is not gated off), and records every ring's
// state at the start of that block, bs. With state_mid it runs on to the first
// block of the unit's second half, bmid = bs + (nblk - bs + 1) / 2, and records the
// state there too. The launch kernels resume from these with the same arithmetic
// (the same warps hold the same rings, so even the warp-uniform choices agree), so
// their results are those of a run from l0. Units in which no ring contributes get
// bstart = their block count.
template <int NDER, bool SPIN2>
__global__ void __launch_bounds__(kComputeThreads) tcstart_kernel(TcDesc D, int *__restrict__ bstart,
                                                                   float *__restrict__ state,
                                                                   float *__restrict__ state_mid) {
  constexpr int NJ = NDER + 1;
  const int rblk = blockIdx.x, m = blockIdx.y, tid = threadIdx.x;
  const int l0 = unit_l0(m, SPIN2);
  const int nblk = (D.lmax >= l0) ? (D.lmax - l0 + 8) / 8 : 0;
  const long long b0 = D.blk[m];
  const long long unit = (long long)m * D.nrblk + rblk;
  bool active;
  const int r = unit_ring<SPIN2>(D, rblk, tid, active);
  Leib<float, NDER> LC;
  leibniz_coefs<float, NDER>(D.rt.z[r], D.rt.sint[r], 1.0 / (double)(D.lmax + 1), LC);
  float a[NJ], b[NJ];
  int sc;
  unit_seed<NDER, SPIN2>(D, r, m, active, a, b, sc);
  const float w = (float)D.rt.omza[r];
  const bool mirror = SPIN2 && tid >= 64;
  const int qo = mirror ? 4 : 2;
  const size_t so = (size_t)unit * (2 * NJ + 1) * kComputeThreads + tid;
  int first = nblk, stop = nblk;
  for (int blk = 0; blk < stop; ++blk) {
    const float4 *stp = (const float4 *)(D.step + (b0 + blk) * step_stride(SPIN2));
    const float4 A0 = __ldg(stp), A1 = __ldg(stp + 1);
    const float4 C0 = __ldg(stp + qo), C1 = __ldg(stp + qo + 1);
    const float Av[8] = {A0.x, A0.y, A0.z, A0.w, A1.x, A1.y, A1.z, A1.w};
    const float Cv[8] = {C0.x, C0.y, C0.z, C0.w, C1.x, C1.y, C1.z, C1.w};
    float sa[NJ], sb[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      sa[j] = a[j];
      sb[j] = b[j];
    }
    const int ssc = sc;
    float buf0[NJ][4], buf1[NJ][4];
    block_steps<NDER, SPIN2>(mirror, a, b, sc, LC, w, Av, Cv, buf0, buf1);
    // a ring can have contributed in this block only if its scale is 0 at the end
    if (first == nblk && __syncthreads_or(sc == 0)) {
      first = blk;
      float *st = state + so;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        st[j * kComputeThreads] = sa[j];
        st[(NJ + j) * kComputeThreads] = sb[j];
      }
      st[2 * NJ * kComputeThreads] = __int_as_float(ssc);
      if (!state_mid) break;
      stop = first + (nblk - first + 1) / 2;  // bmid: record the state at its start
    }
  }
  if (state_mid && first < nblk) {
    // (a, b, sc) are now the state at the start of block `stop` = bmid
    float *st = state_mid + so;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      st[j * kComputeThreads] = a[j];
      st[(NJ + j) * kComputeThreads] = b[j];
    }
    st[2 * NJ * kComputeThreads] = __int_as_float(sc);
  }
  if (tid == 0) bstart[unit] = first;
}

// ---------------------------------------------------------------------------
// plan-time and per-call tables

// step factors per block (layout of step_stride): A_{l+1} (8 floats), then for spin 0
// A - 2 (8 floats), for spin 2 Qn = A - 2 + A C and Qs = A - 2 - A C (8 each), with
// C = m s/(l(l+1)), formed in double from the plan's {k_l, A_{l+1} - 2}; 0 past lmax
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
  float A = 0.0f, qn = 0.0f, qs = 0.0f;
  if (l <= lmax) {
    const double Am2 = (double)tab[(long long)m * (2 * lmax + 1 - m) / 2 + l].y, Ad = 2.0 + Am2;
    const double C = (s == 0) ? 0.0 : (double)m * s / ((double)l * (l + 1.0));  // spin 0 has l = 0
    A = (float)Ad;
    qn = (float)(Am2 + Ad * C);
    qs = (float)(Am2 - Ad * C);
  }
  float *o = out + (blkofs[m] + blk) * step_stride(as == 2);
  o[k] = A;
  o[8 + k] = qn;
  if (as == 2) o[16 + k] = qs;
}

// Coefficient tiles per 8-l block: B[n][k] for column n = 4 rho + c (n < NC) and
// l = l0 + 8 blk + k, as TF32 hi (first NC x 32 bytes) and lo (next), K-major
// without swizzle. BF16x3 (bf16 != 0): the first half holds B[n][k] for k < 16 with
// the BF16 hi of l0 + 8 blk + (k mod 8), the second half the same with the lo parts,
// matching the basis tile [hi | lo] along K.
//   spin 2: c = 0,1: k_l (E + iB) re, im;  c = 2,3: k_l (-1)^(l+m) (E - iB) re, im
//   spin 0: c = 0,1: k_l a re, im;         c = 2,3: k_l (-1)^(l+m) a re, im
struct TcAlm {
  const double *a[kMaxReal];  // spin 0 field, or E (spin 2)
  const double *b[kMaxReal];  // B (spin 2), may be NULL
};

// One warp per (8-l block, 32 columns) (blocks of all m numbered contiguously; the
// block's m from the plan's block table); lane n owns column 32 h + n: it forms the
// column's 8 values and writes their hi and lo parts as 16-byte vectors.
__global__ void __launch_bounds__(256) tcprep_kernel(int lmax, int s, int nreal, int nc, int bf16, TcAlm alm,
                                                     const long long *__restrict__ blkofs,
                                                     const int *__restrict__ blkm, long long nblocks,
                                                     const float2 *__restrict__ tab, unsigned char *__restrict__ out) {
  const int groups = nc >> 5;
  const long long W = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const long long B = W / groups;
  if (B >= nblocks) return;
  const int n = (int)(W - B * groups) * 32 + (threadIdx.x & 31);
  const int m = __ldg(blkm + B);
  const int blk = (int)(B - blkofs[m]);
  const int as = s < 0 ? -s : s;
  const int l0 = m > as ? m : as;
  const int rho = n >> 2, c = n & 3;
  float hv[8], lv[8];
  // the coefficients are taken to float once and scaled in float: the tiles hold
  // float (split) values, and double arithmetic would queue on the slow FP64 pipe
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int l = l0 + 8 * blk + k;
    float v = 0.0f;
    if (l <= lmax && rho < nreal) {
      const long long idx = (long long)m * (2 * lmax + 1 - m) / 2 + l;
      const float kl = tab[idx].x;
      const float sg = ((l + m) & 1) ? -1.0f : 1.0f;
      const double *A = alm.a[rho], *Bm = alm.b[rho];
      const float ar = (float)A[2 * idx], ai = (m > 0) ? (float)A[2 * idx + 1] : 0.0f;
      if (s == 0) {
        const float re = ar * kl, im = ai * kl;
        v = (c == 0) ? re : (c == 1) ? im : (c == 2) ? sg * re : sg * im;
      } else {
        const float br = Bm ? (float)Bm[2 * idx] : 0.0f, bi = (Bm && m > 0) ? (float)Bm[2 * idx + 1] : 0.0f;
        v = (c == 0) ? (ar - bi) * kl : (c == 1) ? (ai + br) * kl : (c == 2) ? sg * kl * (ar + bi) : sg * kl * (ai - br);
      }
    }
    if (bf16) {
      hv[k] = v;
    } else {
      hv[k] = __uint_as_float(to_tf32(v));
      lv[k] = __uint_as_float(to_tf32(v - hv[k]));
    }
  }
  const uint32_t half = btile_bytes(nc) / 2;
  unsigned char *o = out + B * (2 * half);
  if (bf16) {
    uint4 h, l;
    bf16_split2(hv[0], hv[1], h.x, l.x);
    bf16_split2(hv[2], hv[3], h.y, l.y);
    bf16_split2(hv[4], hv[5], h.z, l.z);
    bf16_split2(hv[6], hv[7], h.w, l.w);
    *(uint4 *)(o + can_off(n, 0)) = h;  // k = 0..7 (against the basis hi)
    *(uint4 *)(o + can_off(n, 4)) = h;  // k = 8..15 (against the basis lo)
    *(uint4 *)(o + half + can_off(n, 0)) = l;
    *(uint4 *)(o + half + can_off(n, 4)) = l;
    return;
  }
  *(float4 *)(o + can_off(n, 0)) = make_float4(hv[0], hv[1], hv[2], hv[3]);
  *(float4 *)(o + can_off(n, 4)) = make_float4(hv[4], hv[5], hv[6], hv[7]);
  *(float4 *)(o + half + can_off(n, 0)) = make_float4(lv[0], lv[1], lv[2], lv[3]);
  *(float4 *)(o + half + can_off(n, 4)) = make_float4(lv[4], lv[5], lv[6], lv[7]);
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
  const int nc = tc_cols(p->tc_nder);
  if (nreal < 1 || nreal > nc / 4) return cudaErrorInvalidValue;
  TcAlm alm;
  for (int i = 0; i < kMaxReal; ++i) {
    alm.a[i] = (i < nreal) ? a[i] : nullptr;
    alm.b[i] = (i < nreal && b) ? b[i] : nullptr;
  }
  const long long nblocks = (s == 2) ? p->tc_nblk2 : p->tc_nblk0;
  if (nblocks == 0) return cudaSuccess;
  const long long warps = nblocks * (nc / 32);
  tcprep_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(p->lmax, s, nreal, nc,
                                                             tc_mode(p->precision) == kModeBf16x3 ? 1 : 0, alm,
                                                             blkofs, (s == 2) ? p->tc_bm2 : p->tc_bm0, nblocks,
                                                             (const float2 *)tab,
                                                             (unsigned char *)out);
  return cudaGetLastError();
}

// Realisations per launch and coefficient-tile bytes per block at a plan's order.
int tc_realisations(int nder) { return tc_cols(nder) / 4; }
size_t tc_btile_bytes(int nder) { return btile_bytes(tc_cols(nder)); }
// Rings per CTA: spin 2 takes 64 north rings with their mirrors, spin 0 128 north rings.
int tc_ring_blocks(const tl_plan *p, int spin) {
  return spin == 2 ? (2 * p->nside + 63) / 64 : (2 * p->nside + 127) / 128;
}

// Dynamic shared memory: two coefficient tiles and the spin-2 exchange area, raised
// to the size that keeps the CTAs per SM within the tensor memory (512 columns per
// SM): 4 CTAs (46 KB), 2 (76 KB) or 1 (114 KB).
template <int CTAS, int NC, int NH> static size_t umma_smem() {
  const size_t floor_b = CTAS >= 4 ? 46 * 1024 : CTAS == 2 ? 76 * 1024 : 114 * 1024;
  const size_t need = xch_offset<NC, NH>() + kXchBytes;
  return need > floor_b ? need : floor_b;
}

// which: 0 temperature, 1 lensing potential, 2 polarisation (its start table)
static TcDesc make_desc(const tl_plan *p, int which, int nreal, const void *btiles, void *d7a, void *d7b,
                        long long rstride) {
  const int spin = which == 2 ? 2 : 0;
  TcDesc D;
  memset(&D, 0, sizeof D);
  D.rt = p->ring;
  D.lnorm0 = p->lnorm0;
  D.nside = p->nside;
  D.lmax = p->lmax;
  D.mmax = p->mmax;
  D.nrings = p->nrings;
  D.nreal = nreal;
  D.blk = spin == 2 ? p->tc_blk2 : p->tc_blk0;
  D.step = spin == 2 ? p->tc_step2 : p->tc_step0;
  D.b = (const unsigned char *)btiles;
  D.d7a = (float2 *)d7a;
  D.d7b = (float2 *)d7b;
  D.rstride = rstride;
  D.prows = d7_rows_il(p->nrings);
  D.err = p->dev_err;
  D.nrblk = tc_ring_blocks(p, spin);
  D.bstart = which == 2 ? p->tc_bs2 : which == 1 ? p->tc_bsp : p->tc_bs0;
  D.state = which == 2 ? p->tc_st2 : which == 1 ? p->tc_stp : p->tc_st0;
  D.state_mid = which == 2 ? p->tc_sm2 : which == 1 ? p->tc_smp : p->tc_sm0;
  D.polls = p->wait_polls > 0 ? p->wait_polls : (1 << 24);
  D.stall = p->wait_stall;
  if (!D.state) D.bstart = nullptr;  // no table: every unit starts at l0
  if (!D.bstart) D.state_mid = nullptr;
  return D;
}

// Write the descriptor of a plan's work for nreal realisations to dst: which = 0
// temperature, 1 lensing potential, 2 polarisation.
void tc_desc_write(const tl_plan *p, int which, int nreal, void *dst) {
  const TcDesc d = which == 2   ? make_desc(p, 2, nreal, p->tc_b2, p->d7_Q, p->d7_U, p->d7_rstride)
                   : which == 1 ? make_desc(p, 1, nreal, p->tc_bp, p->d7_P, nullptr, p->d7p_rstride)
                                : make_desc(p, 0, nreal, p->tc_b0, p->d7_T, nullptr, p->d7_rstride);
  memcpy(dst, &d, sizeof d);
}
size_t tc_desc_bytes() { return sizeof(TcDesc); }

template <typename K>
static cudaError_t set_smem(K kernel, size_t smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int NDER, int MODE>
static cudaError_t u2(const tl_plan *p, int nreal, void *dq, void *du, long long rstride, cudaStream_t s) {
  typedef Tc<NDER, MODE> C;
  const size_t smem = umma_smem<C::TM::ctas, C::NC, C::NH>();
  TL_CUDA_TRY(set_smem(legendre_spin2_umma<NDER, MODE>, smem));
  dim3 grid(tc_ring_blocks(p, 2), p->mmax + 1);
  legendre_spin2_umma<NDER, MODE>
      <<<grid, umma_threads(C::NH), smem, s>>>(make_desc(p, 2, nreal, p->tc_b2, dq, du, rstride));
  return cudaGetLastError();
}

template <int NDER, int CNC, int MODE>
static cudaError_t u0(const tl_plan *p, int which, int nreal, void *d7, long long rstride, cudaStream_t s) {
  typedef Tc0<NDER, MODE, CNC> C;
  const size_t smem = umma_smem<C::TM::ctas, CNC, C::NH>();
  TL_CUDA_TRY(set_smem(legendre_spin0_umma<NDER, MODE, CNC>, smem));
  dim3 grid(tc_ring_blocks(p, 0), p->mmax + 1);
  legendre_spin0_umma<NDER, MODE, CNC><<<grid, umma_threads(C::NH), smem, s>>>(
      make_desc(p, which, nreal, which == 1 ? p->tc_bp : p->tc_b0, d7, nullptr, rstride));
  return cudaGetLastError();
}

template <int NDER, int MODE>
static cudaError_t up(const void *descs, const void *items, int nitems, int *counter, int grid, cudaStream_t s) {
  typedef Tc<NDER, MODE> C;
  const size_t smem = umma_smem<C::TM::ctas, C::NC, C::NH>();
  TL_CUDA_TRY(set_smem(legendre_umma_persistent<NDER, MODE>, smem));
  legendre_umma_persistent<NDER, MODE>
      <<<grid, umma_threads(C::NH), smem, s>>>((const TcDesc *)descs, (const int4 *)items, nitems, counter);
  return cudaGetLastError();
}

#define TL_TC_ORDERS(X) X(1) X(2) X(3) X(4) X(5) X(6)

// the kernel instance of contraction form `mode` (kModeTf32, kModeTf32x3, kModeBf16x3)
#define TL_TC_BY_MODE(mode, F, ...)                                          \
  ((mode) == kModeTf32x3   ? F<__VA_ARGS__, kModeTf32x3>                     \
   : (mode) == kModeBf16x3 ? F<__VA_ARGS__, kModeBf16x3>                     \
                           : F<__VA_ARGS__, kModeTf32>)

cudaError_t launch_legendre_tc_persistent(int nder, int precision, const void *descs, const void *items, int nitems,
                                          int *counter, int grid, cudaStream_t s) {
  const int mode = tc_mode(precision);
  switch (nder) {
#define CASE(n) \
  case n: return TL_TC_BY_MODE(mode, up, n)(descs, items, nitems, counter, grid, s);
    TL_TC_ORDERS(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_legendre_spin2_tc(const tl_plan *p, int nder, int nreal, void *dq, void *du, long long rstride,
                                     cudaStream_t s) {
  if (nder != p->tc_nder) return cudaErrorInvalidValue;
  const int mode = tc_mode(p->precision);
  switch (nder) {
#define CASE(n) \
  case n: return TL_TC_BY_MODE(mode, u2, n)(p, nreal, dq, du, rstride, s);
    TL_TC_ORDERS(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

// which = 0: the temperature at the plan's tc_nder; 1: the lensing potential at
// NDER = 1. The columns are the plan's either way (its coefficient tiles have that width).
cudaError_t launch_legendre_spin0_tc(const tl_plan *p, int which, int nreal, void *d7, long long rstride,
                                     cudaStream_t s) {
  const int mode = tc_mode(p->precision);
  const int nc = tc_cols(p->tc_nder);
  if (which == 1) {
    if (nc == 64) return TL_TC_BY_MODE(mode, u0, 1, 64)(p, 1, nreal, d7, rstride, s);
    return TL_TC_BY_MODE(mode, u0, 1, 32)(p, 1, nreal, d7, rstride, s);
  }
  if (which != 0) return cudaErrorInvalidValue;
  switch (p->tc_nder) {
#define CASE(n) \
  case n: return TL_TC_BY_MODE(mode, u0, n, tc_cols(n))(p, 0, nreal, d7, rstride, s);
    TL_TC_ORDERS(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

// Fill a start table (plan time): which as in make_desc; units of that spin.
cudaError_t launch_tcstart(const tl_plan *p, int which, int *bstart, float *state, float *state_mid,
                           cudaStream_t s) {
  TcDesc D = make_desc(p, which, 1, nullptr, nullptr, nullptr, 0);
  D.bstart = nullptr;
  D.state = nullptr;
  D.state_mid = nullptr;
  const int spin = which == 2 ? 2 : 0;
  const int nder = which == 1 ? 1 : p->tc_nder;
  dim3 grid(tc_ring_blocks(p, spin), p->mmax + 1);
  switch (nder) {
#define CASE(n)                                                                                      \
  case n:                                                                                            \
    if (spin == 2)                                                                                   \
      tcstart_kernel<n, true><<<grid, kComputeThreads, 0, s>>>(D, bstart, state, state_mid);         \
    else                                                                                             \
      tcstart_kernel<n, false><<<grid, kComputeThreads, 0, s>>>(D, bstart, state, state_mid);        \
    return cudaGetLastError();
    TL_TC_ORDERS(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

// Start-table bytes: the state of 128 rings (2 NJ + 1 words each) per unit.
size_t tc_start_state_bytes(const tl_plan *p, int which) {
  const int nj = (which == 1 ? 1 : p->tc_nder) + 1;
  const size_t units = (size_t)(p->mmax + 1) * tc_ring_blocks(p, which == 2 ? 2 : 0);
  return units * (2 * nj + 1) * kComputeThreads * sizeof(float);
}
// Whether the kernels that run a start table's units split them into two halves
// (and so need its midpoint table): which as in make_desc.
bool tc_split(const tl_plan *p, int which) {
  const int mode = tc_mode(p->precision), nc = tc_cols(p->tc_nder);
  if (which == 1) return true;  // the potential's map (2 orders) always has room
  return tc_halves(p->tc_nder + 1, mode, nc) == 2;
}
size_t tc_start_units(const tl_plan *p, int which) {
  return (size_t)(p->mmax + 1) * tc_ring_blocks(p, which == 2 ? 2 : 0);
}

// CTAs per SM that the persistent kernel's tensor memory allows (for the grid size).
int tc_persistent_ctas(int nder, int precision) {
  const int mode = tc_mode(precision);
  switch (nder) {
#define CASE(n)                                                   \
  case n:                                                         \
    return mode == kModeTf32x3   ? Tc<n, kModeTf32x3>::TM::ctas   \
           : mode == kModeBf16x3 ? Tc<n, kModeBf16x3>::TM::ctas   \
                                 : Tc<n, kModeTf32>::TM::ctas;
    TL_TC_ORDERS(CASE)
#undef CASE
  }
  return 1;
}

}  // namespace tl
