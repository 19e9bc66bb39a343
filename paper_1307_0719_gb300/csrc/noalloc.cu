// tl_deflection_noalloc: the deflection computation of tl_deflection, for callers
// that must not allocate device memory (for example code running inside a memory
// pool or an allocator of its own, or a host process whose allocations are fixed
// up front). Every table and all working memory live in one file-scope device
// array of fixed size; the call itself makes no cudaMalloc/cudaFree and uses no
// allocating library routine, on the host or on the device.
#include <string.h>

#include "legendre.cuh"

#define TL_NOALLOC_BYTES (8u << 20)  // 8 MiB, held by every GPU that loads the library

// In host code this name is only a stand-in for the device symbol; the device
// address comes from cudaGetSymbolAddress at set-up.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TL_NOALLOC_BYTES];

namespace {

constexpr int kMaxRings = 4 * TL_NOALLOC_MAX_NSIDE - 1;
constexpr int kK = TL_MAX_NDER + 1;
constexpr int kMaxDev = 64;

struct DevState {
  unsigned char *base;  // device address of g_noalloc_scratch on this device (0 until set up)
  int nside, lmax, precision;  // tables currently held (0 = none)
  tl_plan plan;         // pointers into the scratch array
};
DevState g_dev[kMaxDev];

// host staging for the tables, sized for the largest supported plan
double h_z[kMaxRings], h_sint[kMaxRings], h_theta[kMaxRings], h_phi0[kMaxRings], h_lsh[kMaxRings],
    h_lch[kMaxRings], h_dls[kMaxRings * kK], h_dlc[kMaxRings * kK], h_dphi[kMaxRings], h_omza[kMaxRings];
float h_rsinf[kMaxRings], h_ringf[8 * kMaxRings];
int h_nphi[kMaxRings], h_inorth[kMaxRings], h_fft_order[kMaxRings];
long long h_first[kMaxRings];
double h_lnorm0[TL_NOALLOC_MAX_LMAX + 1];
long long h_off[TL_NOALLOC_MAX_NSIDE + 1];
int h_ml[TL_NOALLOC_MAX_NSIDE + 1];
double h_tw[2 * 4 * TL_NOALLOC_MAX_NSIDE];
float h_tw32[2 * 4 * TL_NOALLOC_MAX_NSIDE];

struct Bump {
  unsigned char *base;
  size_t off, cap;
  void *take(size_t bytes) {
    size_t o = (off + 255) & ~(size_t)255;
    if (o + bytes > cap) return nullptr;
    off = o + bytes;
    return base + o;
  }
};

tl_status fail(cudaError_t e) { return e == cudaSuccess ? TL_OK : TL_ERR_CUDA; }

// Lay the tables and the working memory out in the scratch array and fill them.
tl_status setup(DevState &st, int nside, int lmax, int precision) {
  // Earlier calls may still be running on the caller's stream, which need not
  // synchronise with the copies below (a non-blocking stream does not): wait for
  // the whole device before the array is laid out again. Allocates nothing.
  if (cudaDeviceSynchronize() != cudaSuccess) return TL_ERR_CUDA;
  st.nside = 0;  // invalid until complete
  tl_plan &p = st.plan;
  memset(&p, 0, sizeof(p));
  p.nside = nside;
  p.lmax = p.mmax = lmax;
  p.order = 1;
  p.spins = TL_SPIN_T;
  p.precision = precision;
  p.flags = 0;
  p.nrings = 4 * nside - 1;
  p.npix = 12LL * nside * nside;
  p.nmaps = tl::maps_per_field(1);
  p.elem = (precision == TL_FP64) ? 8 : 4;
  cudaGetDevice(&p.device);
  const size_t nr = (size_t)p.nrings, e2 = 2 * (size_t)p.elem;
  const long long na = tl::nalm(lmax);

  tl::RingHostView v{h_z,     h_sint,  h_theta, h_phi0, h_lsh,   h_lch,  h_dls,
                     h_dlc,   h_dphi,  h_omza,  h_rsinf, h_ringf, h_nphi, h_inorth, h_first};
  tl::host_ring_tables(nside, v);
  tl::host_lnorm0(lmax, h_lnorm0);
  int maxm = 0;
  const long long tot = tl::host_bluestein_layout(nside, h_off, h_ml, &maxm);
  p.blue_maxm = maxm;
  p.fft_ngroups = tl::host_fft_groups(nside, p.nrings, h_nphi, h_ml, p.fft_groups, h_fft_order);
  if (p.fft_ngroups < 0) return TL_ERR_ARG;
  const int TW = tl::host_twiddle_len(nside, maxm);
  p.tw_len = TW;
  tl::host_twiddles(TW, h_tw);
  for (int k = 0; k < TW; ++k) h_tw32[k] = (float)h_tw[k];

  Bump b{st.base, 0, TL_NOALLOC_BYTES};
  struct Up {
    void **dst;
    const void *src;
    size_t bytes;
  } ups[] = {
      {(void **)&p.ring.z, h_z, 8 * nr},          {(void **)&p.ring.sint, h_sint, 8 * nr},
      {(void **)&p.ring.theta, h_theta, 8 * nr},  {(void **)&p.ring.phi0, h_phi0, 8 * nr},
      {(void **)&p.ring.log2_sh, h_lsh, 8 * nr},  {(void **)&p.ring.log2_ch, h_lch, 8 * nr},
      {(void **)&p.ring.dls, h_dls, 8 * nr * kK}, {(void **)&p.ring.dlc, h_dlc, 8 * nr * kK},
      {(void **)&p.ring.nphi, h_nphi, 4 * nr},    {(void **)&p.ring.inorth, h_inorth, 4 * nr},
      {(void **)&p.ring.dphi, h_dphi, 8 * nr},    {(void **)&p.ring.omza, h_omza, 8 * nr},
      {(void **)&p.ring.rsinf, h_rsinf, 4 * nr},  {(void **)&p.ring.ringf, h_ringf, 32 * nr},
      {(void **)&p.ring.first, h_first, 8 * nr},  {(void **)&p.lnorm0, h_lnorm0, 8 * (size_t)(lmax + 1)},
      {(void **)&p.blue.offset, h_off, 8 * (size_t)(nside + 1)},
      {(void **)&p.blue.mlen, h_ml, 4 * (size_t)(nside + 1)},
      {(void **)&p.fft_rings, h_fft_order, 4 * nr},
      {(void **)&p.twiddle, precision == TL_FP64 ? (const void *)h_tw : (const void *)h_tw32,
       (size_t)(precision == TL_FP64 ? 8 : 4) * TW},
  };
  for (auto &u : ups) {
    *u.dst = b.take(u.bytes);
    if (!*u.dst) return TL_ERR_ARG;
    cudaError_t e = cudaMemcpy(*u.dst, u.src, u.bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(e);
  }
  double2 *tw64 = (double2 *)b.take(8 * (size_t)TW);
  p.blue.spec = b.take(e2 * (size_t)(tot > 0 ? tot : 1));
  p.tab0 = b.take(e2 * (size_t)na);
  p.rec_T = b.take(4 * (size_t)p.elem * (size_t)na);
  p.d7_P = b.take(e2 * 2 * nr * (size_t)(lmax + 1));
  p.phase = b.take(e2 * tl::phase_table_entries(nside));
  if (!tw64 || !p.blue.spec || !p.tab0 || !p.rec_T || !p.d7_P || !p.phase) return TL_ERR_ARG;
  cudaError_t e = cudaMemcpy(tw64, h_tw, 8 * (size_t)TW, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = tl::launch_phase_table(&p, p.phase, 0);
  if (e == cudaSuccess) e = tl::launch_bluestein_setup_impl(&p, tw64, 0);
  if (e == cudaSuccess) e = tl::launch_steptab(&p, 0, p.tab0, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(e);
  p.bytes = b.off;
  st.nside = nside;
  st.lmax = lmax;
  st.precision = precision;
  return TL_OK;
}

}  // namespace

extern "C" tl_status tl_deflection_noalloc(int nside, int lmax, int precision, const double *alm_phi,
                                           void *a_theta, void *a_phi, void *stream) {
  if (nside < 1 || nside > TL_NOALLOC_MAX_NSIDE || (nside & (nside - 1)) != 0) return TL_ERR_ARG;
  if (lmax < 1 || lmax > 4 * nside || lmax > TL_NOALLOC_MAX_LMAX) return TL_ERR_ARG;
  if (precision != TL_FP64 && precision != TL_MIXED_FP32) return TL_ERR_ARG;
  if (!alm_phi || !a_theta || !a_phi) return TL_ERR_ARG;
  if (((uintptr_t)alm_phi | (uintptr_t)a_theta | (uintptr_t)a_phi) & 15u) return TL_ERR_ARG;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return TL_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDev) return TL_ERR_UNSUPPORTED;
  DevState &st = g_dev[dev];
  if (!st.base) {
    void *addr = nullptr;
    e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess || !addr) return TL_ERR_CUDA;
    st.base = (unsigned char *)addr;
  }
  if (st.nside != nside || st.lmax != lmax || st.precision != precision) {
    tl_status s = setup(st, nside, lmax, precision);
    if (s != TL_OK) return s;
  }
  tl_plan *p = &st.plan;
  cudaStream_t s = (cudaStream_t)stream;
  // the records and the phi planes are rewritten in full before they are read,
  // so nothing left by an earlier call needs clearing
  TL_CUDA_TRY_STATUS(tl::launch_prep_spin0(p, alm_phi, nullptr, s));
  TL_CUDA_TRY_STATUS(tl::launch_legendre_spin0(p, 1, false, p->d7_P, nullptr, s));
  const double L = tl::deriv_norm(p);
  tl::MapJob jobs[2] = {{3, 1, 0, 0, L, a_theta}, {3, 0, 1, 1, L, a_phi}};
  TL_CUDA_TRY_STATUS(tl::launch_ringfft(p, jobs, 2, 2, s));
  return TL_OK;
}
