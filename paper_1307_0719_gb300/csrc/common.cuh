// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/taylens.h"

#define TL_MAX_ORDER 6
// largest plan tl_deflection_noalloc serves from its fixed device array
#define TL_NOALLOC_MAX_NSIDE 128
#define TL_NOALLOC_MAX_LMAX 256
#define TL_MAX_NDER 6
#define TL_MAX_BATCH 16  // realisations per tensor-core Legendre launch at most  // highest theta-derivative order a Legendre kernel carries

namespace tl {

// ---------------------------------------------------------------------------
// HEALPix RING geometry (Gorski et al. 2005), one entry per ring r = 0 .. 4N-2
// (ring number r+1 counted from the north pole).
struct RingTable {
  double *z;       // cos(theta)
  double *sint;    // sin(theta)
  double *theta;   // colatitude
  double *phi0;    // longitude of the ring's first pixel
  double *dphi;    // 2 pi / nphi: longitude step between the ring's pixels
  double *omza;    // 1 - |cos(theta)|, formed without cancellation
  float *rsinf;    // 1 / sin(theta), rounded to float (single-precision kernels)
  float *ringf;    // [ring][8] for the float gather: z, sin, 1 - |z|, theta hi, theta lo (hi + lo = theta)
  double *log2_sh; // log2 sin(theta/2)
  double *log2_ch; // log2 cos(theta/2)
  double *dls;     // [ring][k], k = 1..TL_MAX_NDER+1: d^k/dtheta^k ln sin(theta/2)
  double *dlc;     // [ring][k]: d^k/dtheta^k ln cos(theta/2)
  int *nphi;       // pixels in the ring (4 i in the caps, 4 N in the belt)
  int *inorth;     // ring number counted from the nearer pole
  long long *first;// index of the ring's first pixel
};

// Bluestein chirp spectra for the non-power-of-two sub-transform lengths.
struct BluesteinTable {
  void *spec;          // concatenated spectra (T2 of the plan's precision)
  long long *offset;   // [nside]: offset of length i's spectrum, -1 if i is a power of two
  int *mlen;           // [nside]: its FFT length M (power of two >= 2i-1)
};

struct StageTimer;

// Rings of one ring-FFT launch: the equatorial belt, the power-of-two caps, or
// the caps whose Bluestein length is M; ring indices fft_rings[first .. first + count),
// largest first. Each launch gets the shared memory its own rings need.
struct FftGroup {
  int first, count, ni_max, ni_min, M;
};
#define TL_MAX_FFT_GROUPS 24

}  // namespace tl

struct tl_plan {
  int nside, lmax, mmax, order, spins, precision, flags;
  int lmax_phi;          // band limit of the lensing potential (lmax unless set)
  tl_plan *phi_plan;     // its deflection plan when lmax_phi != lmax (else nullptr)
  int nrings;
  long long npix;
  int nmaps;      // maps per field
  int device;
  int elem;       // bytes per map element (8 or 4)
  tl::RingTable ring;
  tl::BluesteinTable blue;
  double *lnorm0;       // [lmax+1] log2 of sqrt((2m+1)/4pi) sqrt(C(2m,m)) (device)
  void *twiddle;        // [TW/2] e^{-2 pi i k / TW} in T2 (device)
  int tw_len;
  int blue_maxm;        // largest Bluestein FFT length (0 if none)
  int blue_reg_lg;      // Bluestein lengths M >= 2^blue_reg_lg (up to 2^12) run the register passes and keep
                        // their spectra in natural order (0: none; bit-reversed order for the others)
  int fft_batch;        // Bluestein sub-transforms run together in the ring FFT (1 or 4; 0 = choose)
  int ring_reg;         // single precision: register-pass ring FFT where a group allows it (1, default) or not (0)
  int *fft_rings;       // ring indices grouped by FFT launch (device)
  int fft_ngroups;
  tl::FftGroup fft_groups[TL_MAX_FFT_GROUPS];
  // workspace
  void *tab0, *tab2;    // plan-time step tables {k_l, A_{l+1}} for spin 0 and spin 2
  void *rec_T, *rec_P, *rec_QU; // coefficient records
  void *d7_T, *d7_Q, *d7_U, *d7_P; // per-ring Fourier coefficients [j][ring][m] (T2)
  // tensor-core Legendre stage (TL_MIXED_TF32, TL_MIXED_TF32x3, TL_MIXED_BF16x3): blocks of 8 l per m
  int batch;             // realisations sharing one Legendre launch (1, or 8 on tensor cores)
  int tc_nder;           // derivative orders carried there (max(order, 1))
  long long *tc_blk0, *tc_blk2;   // [lmax+1] first block of each m (spin 0 / spin 2)
  int *tc_bm0, *tc_bm2;           // [blocks] the m of each block (spin 0 / spin 2)
  long long tc_nblk0, tc_nblk2;   // blocks in all
  // start tables (T, potential, Q/U): first contributing block per unit and the
  // recurrence state there
  int *tc_bs0, *tc_bsp, *tc_bs2;
  float *tc_st0, *tc_stp, *tc_st2;
  float *tc_sm0, *tc_smp, *tc_sm2;  // the same state at each unit's midpoint block (split units)
  float *tc_step0, *tc_step2;     // per 8-l block: A_{l+1} x 8, then A - 2 x 8 (spin 0) or Qn, Qs x 8 (spin 2)
  void *tc_b0, *tc_bp, *tc_b2;    // [blocks] 2 KB coefficient tiles (TF32 hi, lo; 32 columns x 8 l)
  int *dev_err;                   // set by a kernel whose bounded wait timed out
  long long d7_rstride, d7p_rstride;  // T2 elements between realisations' D7 planes
  void *d3;            // derivative maps [3*nmaps][npix] (T), Taylor-ready
  void *phase;          // ring-FFT phase table e^{i pi t / (4 ni)} per quarter length ni (T2)
  int *gq;             // float plans: pixels the float gather defers to the double pass [npix]
  int *gq_count;       // their number (reset before every gather)
  int num_sms;         // multiprocessors of the plan's device
  int wait_polls;      // polls of a tensor-core mbarrier wait (0: the default, 2^24)
  int wait_stall;      // self-test of the timeout path (tl_plan_set_wait_limit)
  void *alpha;         // [2][npix] (T)
  void *adj_dbar;      // adjoint: gradients of the derivative maps, as d3 (allocated on first use)
  void *adj_ga;        // adjoint: [2][npix] deflection gradients (allocated on first use)
  void *stage_alm;     // host-path staging: stage_cap x 4 x nalm complex128
  void *stage_out;     // host-path staging: stage_cap x 3 x npix (T)
  int stage_cap;       // realisations the staging holds (0: none yet)
  cudaStream_t copy_stream;                 // host-path copies of finished maps (created on first use)
  cudaEvent_t done_ev[TL_MAX_BATCH];        // a realisation's maps are final (recorded after its gather)
  cudaEvent_t copied_ev;                    // the copy stream's last copy of a call
  int done_rec;                             // lens_stage_after_legendre records done_ev[r] while set
  cudaEvent_t in_ev[3];                     // host path: T staged (compute stream), phi staged, E/B staged
  int in_wait;                              // the tensor-core chunk waits for in_ev[1], in_ev[2] while set
  size_t bytes;
  // optional stage timing
  int timing;
  cudaEvent_t ev[8];
  float stage_ms[7];
  int nstage;
  // per realisation of a tensor-core chunk: before its ring FFTs, after them (before
  // the gather), after the gather; summed into the FFT and gather totals
  cudaEvent_t evr[3 * TL_MAX_BATCH];
  int nevr;
};

namespace tl {

inline long long nalm(int lmax) { return (long long)(lmax + 1) * (lmax + 2) / 2; }
inline int maps_per_field(int order) { return (order + 1) * (order + 2) / 2; }

// kernel launchers (defined in the .cu files)
cudaError_t launch_steptab(const tl_plan *p, int s, void *tab, cudaStream_t st);
// prepares rec_T from alm (if not NULL) and rec_P from alm_phi (if not NULL)
cudaError_t launch_prep_spin0(const tl_plan *p, const double *alm, const double *alm_phi, cudaStream_t s);
cudaError_t launch_prep_spin2(const tl_plan *p, const double *alm_E, const double *alm_B, cudaStream_t s);
cudaError_t launch_legendre_spin0(const tl_plan *p, int nder, bool phi, void *d7, void *d7p, cudaStream_t s);
cudaError_t launch_legendre_spin2(const tl_plan *p, int nder, cudaStream_t s);

// Pixel-tiled layout of the plan's derivative maps (d3): [tile][map][kD3Tile], one
// tile holding every map's values of kD3Tile consecutive pixels, so that the gather's
// reads of all maps at an expansion pixel fall in one 46 KB chunk (one page) instead
// of one page per map; maps = fields x maps per field, T first.
constexpr int kD3TileLg = 8, kD3Tile = 1 << kD3TileLg;
__host__ __device__ __forceinline__ long long d3_tiles(long long npix) { return (npix + kD3Tile - 1) >> kD3TileLg; }
// element of pixel p in the tile layout, relative to a map's own offset m * kD3Tile
__host__ __device__ __forceinline__ long long d3_pix(long long p, long long tile_stride) {
  return (p >> kD3TileLg) * tile_stride + (p & (kD3Tile - 1));
}

// Coefficient planes written by the tensor-core Legendre stage interleave four rings
// per 32-byte sector, element (ring r, order m) at ((r / 4) (mmax + 1) + m) 4 + r mod 4,
// so that a warp of consecutive rings stores whole sectors (a plain [ring][m] row
// would take one partial sector per ring); such a plane has a multiple of 4 rows.
// The SIMT stages and the adjoint keep plain [ring][m] rows.
__host__ __device__ __forceinline__ int d7_rows_il(int nrings) { return (nrings + 3) & ~3; }
__host__ __device__ __forceinline__ size_t d7_il(int r, int m, size_t ld) {
  return ((size_t)(r >> 2) * ld + (size_t)m) * 4 + (size_t)(r & 3);
}

// One output map of the ring FFT stage.
struct MapJob {
  int plane;       // which D7 plane set: 0 = T, 1 = Q, 2 = U, 3 = phi
  int j, k;        // derivative orders
  int div_sint;    // divide by sin(theta) of the ring
  double scale;    // multiplies d_theta^j d_phi^k (after undoing the 1/L^j, L^k normalisation)
  void *out;       // plain: [npix] map; tiled: the map's first element m * kD3Tile of the tile layout
  long long tile;  // 0: plain layout; else elements between tiles (maps x kD3Tile)
  int il;          // the plane's rows are four-ring interleaved (tensor-core stage output)
};
cudaError_t launch_ringfft(const tl_plan *p, const MapJob *jobs, int njobs, int nder_planes,
                           cudaStream_t s);
// as launch_ringfft with explicit plane bases (T, Q, U, phi) for one realisation
cudaError_t launch_ringfft_planes(const tl_plan *p, const void *const *planes, const MapJob *jobs, int njobs,
                                  cudaStream_t s);
// One output plane of the adjoint ring FFT: plane 0..2 (T, Q, U) row j from the
// maps d_theta^j d_phi^k, k < nk, at in + map_index(j, k) npix; plane 3 (phi) row
// j from the single map at in (j = 1: the theta deflection, j = 0: the phi one).
struct AdjMapJob {
  int plane, j, nk;
  const void *in;
};
cudaError_t launch_ringfft_adjoint(const tl_plan *p, void *const *planes, const AdjMapJob *jobs, int njobs,
                                   cudaStream_t s);
cudaError_t launch_legendre_adj0(const tl_plan *p, int nder_T, const void *FT, const void *FP, double *aT,
                                 double *aP, cudaStream_t s);
cudaError_t launch_legendre_adj2(const tl_plan *p, int nder, const void *FQ, const void *FU, double *aE, double *aB,
                                 cudaStream_t s);
cudaError_t launch_adj_finish(const tl_plan *p, double *gT, double *gP, double *gE, double *gB, cudaStream_t s);
cudaError_t launch_gather_adjoint(const tl_plan *p, const void *alpha, const void *d3, const void *gT, const void *gQ,
                                  const void *gU, void *dbar, void *ga, cudaStream_t s);
size_t phase_table_entries(int nside);
cudaError_t launch_phase_table(const tl_plan *p, void *out, cudaStream_t s);
cudaError_t launch_tcstep(const tl_plan *p, int s, const long long *blkofs, const void *tab, float *out,
                          cudaStream_t st);
cudaError_t launch_tcprep(const tl_plan *p, int s, int nreal, const double *const *a, const double *const *b,
                          const long long *blkofs, const void *tab, void *out, cudaStream_t st);
cudaError_t launch_legendre_spin2_tc(const tl_plan *p, int nder, int nreal, void *dq, void *du, long long rstride,
                                     cudaStream_t s);
// spin-0 field (which = 0: temperature at tc_nder, 1: the lensing potential at
// nder = 1) from its coefficient tiles into the planes d7
cudaError_t launch_legendre_spin0_tc(const tl_plan *p, int which, int nreal, void *d7, long long rstride,
                                     cudaStream_t s);
// start tables of the tensor-core Legendre stage (which: 0 T, 1 potential, 2 Q/U)
cudaError_t launch_tcstart(const tl_plan *p, int which, int *bstart, float *state, float *state_mid,
                           cudaStream_t s);
bool tc_split(const tl_plan *p, int which);
size_t tc_start_state_bytes(const tl_plan *p, int which);
size_t tc_start_units(const tl_plan *p, int which);
cudaError_t launch_bluestein_setup(tl_plan *p, cudaStream_t s);
// CTAs per m of the tensor-core Legendre kernels (128 rings each), and the CTAs per
// SM that the persistent kernel's tensor memory allows
int tc_ring_blocks(const tl_plan *p, int spin);
int tc_realisations(int nder);  // realisations per tensor-core Legendre launch at tc_nder
size_t tc_btile_bytes(int nder);  // coefficient-tile bytes per 8-l block
int tc_persistent_ctas(int nder, int precision);
cudaError_t launch_gather(const tl_plan *p, const void *alpha, const void *d3, void *T, void *Q,
                          void *U, cudaStream_t s);

// host table builders (tables.cu); arrays sized by the caller:
// rings: 4 nside - 1 entries (dls, dlc: (4 nside - 1) * (TL_MAX_NDER + 1)),
// lnorm0: lmax + 1, Bluestein off/ml: nside + 1, twiddles: TW doubles
struct RingHostView {
  double *z, *sint, *theta, *phi0, *lsh, *lch, *dls, *dlc, *dphi, *omza;
  float *rsinf, *ringf;
  int *nphi, *inorth;
  long long *first;
};
void host_ring_tables(int nside, const RingHostView &h);
void host_lnorm0(int lmax, double *out);
long long host_bluestein_layout(int nside, long long *off, int *ml, int *maxm);
int host_twiddle_len(int nside, int maxm);
void host_twiddles(int TW, double *tw);
size_t ringfft_smem_bytes(const tl_plan *p);
// ring-FFT launch groups (no allocation): fills groups[] and order[nrings]; returns
// the number of groups, or -1 if there are more than TL_MAX_FFT_GROUPS
int host_fft_groups(int nside, int nrings, const int *nphi, const int *ml, FftGroup *groups, int *order);
cudaError_t launch_bluestein_setup_impl(tl_plan *p, const double2 *tw64, cudaStream_t s);

// normalisation of theta derivatives inside the Legendre stage: lambda^(j) / L^j
inline double deriv_norm(const tl_plan *p) { return (double)(p->lmax + 1); }

}  // namespace tl

#define TL_CUDA_TRY(call)                         \
  do {                                            \
    cudaError_t _e = (call);                      \
    if (_e != cudaSuccess) return _e;             \
  } while (0)

#define TL_CUDA_TRY_STATUS(call)                                                   \
  do {                                                                             \
    cudaError_t _e = (call);                                                       \
    if (_e != cudaSuccess) return _e == cudaErrorMemoryAllocation ? TL_ERR_NOMEM : TL_ERR_CUDA; \
  } while (0)
