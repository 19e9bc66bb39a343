// Plan creation, workspace and the C ABI (taylens.h).
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <utility>
#include <vector>

#include "legendre.cuh"

using namespace tl;

static tl_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return TL_OK;
  if (e == cudaErrorMemoryAllocation) return TL_ERR_NOMEM;
  return TL_ERR_CUDA;
}

#define TRY_CUDA(call)                          \
  do {                                          \
    cudaError_t _e = (call);                    \
    if (_e != cudaSuccess) return from_cuda(_e); \
  } while (0)

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

extern "C" const char *tl_status_string(tl_status s) {
  switch (s) {
    case TL_OK: return "ok";
    case TL_ERR_ARG: return "invalid argument";
    case TL_ERR_NOMEM: return "out of memory";
    case TL_ERR_CUDA: return "CUDA runtime error";
    case TL_ERR_TIMEOUT: return "device wait timed out";
    case TL_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

// ---------------------------------------------------------------------------
// host tables (tables.cu) gathered into vectors

struct HostRings {
  std::vector<double> z, sint, theta, phi0, lsh, lch, dls, dlc, dphi, omza;
  std::vector<float> rsinf, ringf;
  std::vector<int> nphi, inorth;
  std::vector<long long> first;
};

static void build_rings(int N, HostRings &h) {
  const size_t nr = 4 * (size_t)N - 1, K = TL_MAX_NDER + 1;
  h.z.resize(nr); h.sint.resize(nr); h.theta.resize(nr); h.phi0.resize(nr);
  h.lsh.resize(nr); h.lch.resize(nr); h.dls.resize(nr * K); h.dlc.resize(nr * K);
  h.dphi.resize(nr); h.omza.resize(nr); h.rsinf.resize(nr); h.ringf.resize(8 * nr);
  h.nphi.resize(nr); h.inorth.resize(nr); h.first.resize(nr);
  RingHostView v{h.z.data(), h.sint.data(), h.theta.data(), h.phi0.data(), h.lsh.data(), h.lch.data(),
                 h.dls.data(), h.dlc.data(), h.dphi.data(), h.omza.data(), h.rsinf.data(), h.ringf.data(), h.nphi.data(), h.inorth.data(),
                 h.first.data()};
  host_ring_tables(N, v);
}

template <typename V>
static cudaError_t upload(V **dptr, const std::vector<V> &h, size_t *bytes) {
  size_t b = sizeof(V) * (h.empty() ? 1 : h.size());
  cudaError_t e = cudaMalloc((void **)dptr, b);
  if (e != cudaSuccess) return e;
  *bytes += b;
  if (!h.empty()) return cudaMemcpy(*dptr, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice);
  return cudaSuccess;
}

static cudaError_t dalloc(void **p, size_t b, size_t *bytes) {
  cudaError_t e = cudaMalloc(p, b ? b : 16);
  if (e == cudaSuccess) *bytes += b;
  return e;
}

static void free_plan(tl_plan *p) {
  if (!p) return;
  if (p->copy_stream) {
    cudaStreamSynchronize(p->copy_stream);
    for (int i = 0; i < TL_MAX_BATCH; ++i)
      if (p->done_ev[i]) cudaEventDestroy(p->done_ev[i]);
    if (p->copied_ev) cudaEventDestroy(p->copied_ev);
    for (int i = 0; i < 3; ++i)
      if (p->in_ev[i]) cudaEventDestroy(p->in_ev[i]);
    cudaStreamDestroy(p->copy_stream);
    p->copy_stream = nullptr;
  }
  if (p->phi_plan) {
    free_plan(p->phi_plan);
    p->phi_plan = nullptr;
  }
  void *ptrs[] = {p->ring.z, p->ring.sint, p->ring.theta, p->ring.phi0, p->ring.dphi, p->ring.omza, p->ring.rsinf, p->ring.ringf,
                  p->ring.log2_sh, p->ring.log2_ch,
                  p->ring.dls, p->ring.dlc, p->ring.nphi, p->ring.inorth, p->ring.first, p->blue.spec,
                  p->blue.offset, p->blue.mlen, p->lnorm0, p->twiddle, p->tab0, p->tab2, p->rec_T, p->rec_P,
                  p->rec_QU,
                  p->d7_T, p->d7_Q, p->d7_U, p->d7_P, p->d3, p->alpha, p->adj_dbar, p->adj_ga, p->stage_alm,
                  p->stage_out, p->gq, p->gq_count, p->phase,
                  p->tc_blk0, p->tc_blk2, p->tc_bm0, p->tc_bm2, p->tc_step0, p->tc_step2, p->tc_b0, p->tc_bp, p->tc_b2, p->dev_err,
                  p->tc_bs0, p->tc_bsp, p->tc_bs2, p->tc_st0, p->tc_stp, p->tc_st2, p->tc_sm0, p->tc_smp,
                  p->tc_sm2,
                  p->fft_rings};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  if (p->timing)
    for (int i = 0; i < 8; ++i)
      if (p->ev[i]) cudaEventDestroy(p->ev[i]);
  if (p->timing)
    for (int i = 0; i < 3 * TL_MAX_BATCH; ++i)
      if (p->evr[i]) cudaEventDestroy(p->evr[i]);
  free(p);
}

static tl_status create_impl(int nside, int lmax, int order, int spins, int precision, int flags, tl_plan *p) {
  p->nside = nside; p->lmax = lmax; p->mmax = lmax; p->order = order; p->spins = spins;
  p->lmax_phi = lmax;
  p->precision = precision; p->flags = flags;
  p->nrings = 4 * nside - 1;
  p->npix = 12LL * nside * nside;
  p->nmaps = maps_per_field(order);
  p->elem = (precision == TL_FP64) ? 8 : 4;
  TRY_CUDA(cudaGetDevice(&p->device));
  TRY_CUDA(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
  size_t *B = &p->bytes;

  HostRings h;
  build_rings(nside, h);
  TRY_CUDA(upload(&p->ring.z, h.z, B)); TRY_CUDA(upload(&p->ring.sint, h.sint, B));
  TRY_CUDA(upload(&p->ring.theta, h.theta, B)); TRY_CUDA(upload(&p->ring.phi0, h.phi0, B));
  TRY_CUDA(upload(&p->ring.log2_sh, h.lsh, B)); TRY_CUDA(upload(&p->ring.log2_ch, h.lch, B));
  TRY_CUDA(upload(&p->ring.dls, h.dls, B)); TRY_CUDA(upload(&p->ring.dlc, h.dlc, B));
  TRY_CUDA(upload(&p->ring.dphi, h.dphi, B)); TRY_CUDA(upload(&p->ring.omza, h.omza, B));
  TRY_CUDA(upload(&p->ring.rsinf, h.rsinf, B));
  TRY_CUDA(upload(&p->ring.ringf, h.ringf, B));
  TRY_CUDA(upload(&p->ring.nphi, h.nphi, B)); TRY_CUDA(upload(&p->ring.inorth, h.inorth, B));
  TRY_CUDA(upload(&p->ring.first, h.first, B));

  std::vector<double> ln0(lmax + 1);
  host_lnorm0(lmax, ln0.data());
  TRY_CUDA(upload(&p->lnorm0, ln0, B));

  std::vector<long long> off(nside + 1);
  std::vector<int> ml(nside + 1);
  int maxm = 0;
  const long long tot = host_bluestein_layout(nside, off.data(), ml.data(), &maxm);
  p->blue_maxm = maxm;
  TRY_CUDA(upload(&p->blue.offset, off, B));
  TRY_CUDA(upload(&p->blue.mlen, ml, B));
  const size_t e2 = 2 * (size_t)p->elem;
  TRY_CUDA(dalloc(&p->blue.spec, e2 * (size_t)(tot > 0 ? tot : 1), B));

  // ring-FFT launch groups: belt, caps by Bluestein length, power-of-two caps
  {
    std::vector<int> order(p->nrings);
    p->fft_ngroups = host_fft_groups(nside, p->nrings, h.nphi.data(), ml.data(), p->fft_groups, order.data());
    if (p->fft_ngroups < 0) return TL_ERR_UNSUPPORTED;
    TRY_CUDA(upload(&p->fft_rings, order, B));
  }

  // twiddles e^{-2 pi i k / TW}, k < TW/2, for every power-of-two length used
  const int TW = host_twiddle_len(nside, maxm);
  p->tw_len = TW;
  std::vector<double> tw64(TW);  // interleaved (re, im)
  host_twiddles(TW, tw64.data());
  double *dtw64 = nullptr;
  {
    size_t dummy = 0;
    TRY_CUDA(upload(&dtw64, tw64, &dummy));
  }
  if (precision == TL_FP64) {
    TRY_CUDA(dalloc(&p->twiddle, sizeof(double) * TW, B));
    TRY_CUDA(cudaMemcpy(p->twiddle, dtw64, sizeof(double) * TW, cudaMemcpyDeviceToDevice));
  } else {
    std::vector<float> tw32(TW);
    for (int k = 0; k < TW; ++k) tw32[k] = (float)tw64[k];
    TRY_CUDA(upload((float **)&p->twiddle, tw32, B));
  }
  TRY_CUDA(dalloc(&p->phase, e2 * phase_table_entries(nside), B));
  TRY_CUDA(launch_phase_table(p, p->phase, 0));
  const char *rr = getenv("TAYLENS_RING_FFT");  // "shared": the shared-memory kernel for every group
  p->ring_reg = (rr && strcmp(rr, "shared") == 0) ? 0 : 1;
  p->blue_reg_lg = (precision != TL_FP64 && p->ring_reg) ? 11 : 0;
  cudaError_t e = launch_bluestein_setup_impl(p, (const double2 *)dtw64, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(dtw64);
  TRY_CUDA(e);

  // workspace
  const long long na = nalm(lmax);
  const size_t t2 = e2, rec0 = 4 * (size_t)p->elem, rec2 = 8 * (size_t)p->elem;
  const bool pol = (spins & TL_SPIN_QU) != 0;
  const bool tc = (precision == TL_MIXED_TF32 || precision == TL_MIXED_TF32x3 || precision == TL_MIXED_BF16x3);
  // tensor-core plans: the planes' rows rounded up to 4 (the stage writes them four-ring
  // interleaved; the SIMT stages and the adjoint use the first nrings rows plainly)
  const int prows = tc ? d7_rows_il(p->nrings) : p->nrings;
  const size_t plane = (size_t)prows * (p->mmax + 1) * t2;
  p->tc_nder = order > 1 ? order : 1;
  p->batch = tc ? tc_realisations(p->tc_nder) : 1;
  const int nplanes = tc ? p->tc_nder + 1 : order + 1;  // D7 planes per field and realisation
  p->d7_rstride = (long long)nplanes * prows * (p->mmax + 1);
  p->d7p_rstride = 2LL * prows * (p->mmax + 1);
  TRY_CUDA(dalloc(&p->tab0, t2 * na, B));
  TRY_CUDA(launch_steptab(p, 0, p->tab0, 0));
  TRY_CUDA(dalloc(&p->rec_T, rec0 * na, B));
  TRY_CUDA(dalloc(&p->rec_P, t2 * na, B));
  TRY_CUDA(dalloc(&p->d7_T, plane * nplanes * p->batch, B));
  TRY_CUDA(dalloc(&p->d7_P, plane * 2 * p->batch, B));
  if (pol) {
    TRY_CUDA(dalloc(&p->tab2, t2 * na, B));
    TRY_CUDA(launch_steptab(p, 2, p->tab2, 0));
    TRY_CUDA(dalloc(&p->rec_QU, rec2 * na, B));
    TRY_CUDA(dalloc(&p->d7_Q, plane * nplanes * p->batch, B));
    TRY_CUDA(dalloc(&p->d7_U, plane * nplanes * p->batch, B));
  }
  if (tc) {
    // blocks of 8 l per m, from l0 = m (spin 0) or max(m, 2) (spin 2)
    std::vector<long long> b0(lmax + 1), b2(lmax + 1);
    long long n0 = 0, n2 = 0;
    for (int m = 0; m <= lmax; ++m) {
      b0[m] = n0;
      n0 += (lmax - m + 8) / 8;
      b2[m] = n2;
      const int l0 = m > 2 ? m : 2;
      n2 += (lmax >= l0) ? (lmax - l0 + 8) / 8 : 0;
    }
    p->tc_nblk0 = n0;
    p->tc_nblk2 = n2;
    {  // and the m of every block, so that a warp of the tile preparation finds it in one load
      std::vector<int> m0((size_t)n0), m2((size_t)(n2 > 0 ? n2 : 1), 0);
      for (int m = 0; m <= lmax; ++m) {
        for (long long k = b0[m]; k < (m < lmax ? b0[m + 1] : n0); ++k) m0[(size_t)k] = m;
        for (long long k = b2[m]; k < (m < lmax ? b2[m + 1] : n2); ++k) m2[(size_t)k] = m;
      }
      TRY_CUDA(upload(&p->tc_bm0, m0, B));
      if (pol) TRY_CUDA(upload(&p->tc_bm2, m2, B));
    }
    TRY_CUDA(upload(&p->tc_blk0, b0, B));
    TRY_CUDA(dalloc((void **)&p->tc_step0, 64 * (size_t)n0, B));
    TRY_CUDA(launch_tcstep(p, 0, p->tc_blk0, p->tab0, p->tc_step0, 0));
    const size_t bt = tc_btile_bytes(p->tc_nder);
    TRY_CUDA(dalloc(&p->tc_b0, bt * (size_t)n0, B));
    TRY_CUDA(dalloc(&p->tc_bp, bt * (size_t)n0, B));
    if (pol) {
      TRY_CUDA(upload(&p->tc_blk2, b2, B));
      TRY_CUDA(dalloc((void **)&p->tc_step2, 96 * (size_t)(n2 > 0 ? n2 : 1), B));
      TRY_CUDA(launch_tcstep(p, 2, p->tc_blk2, p->tab2, p->tc_step2, 0));
      TRY_CUDA(dalloc(&p->tc_b2, bt * (size_t)(n2 > 0 ? n2 : 1), B));
    }
    // start tables: where each unit's first contribution begins (identical results)
    for (int which = 0; which < (pol ? 3 : 2); ++which) {
      int **bs = which == 0 ? &p->tc_bs0 : which == 1 ? &p->tc_bsp : &p->tc_bs2;
      float **st = which == 0 ? &p->tc_st0 : which == 1 ? &p->tc_stp : &p->tc_st2;
      float **sm = which == 0 ? &p->tc_sm0 : which == 1 ? &p->tc_smp : &p->tc_sm2;
      TRY_CUDA(dalloc((void **)bs, sizeof(int) * tc_start_units(p, which), B));
      TRY_CUDA(dalloc((void **)st, tc_start_state_bytes(p, which), B));
      if (tc_split(p, which)) TRY_CUDA(dalloc((void **)sm, tc_start_state_bytes(p, which), B));
      TRY_CUDA(launch_tcstart(p, which, *bs, *st, *sm, 0));
    }
    TRY_CUDA(cudaDeviceSynchronize());
  }
  TRY_CUDA(dalloc((void **)&p->dev_err, sizeof(int), B));
  TRY_CUDA(cudaMemset(p->dev_err, 0, sizeof(int)));
  const int nfield = pol ? 3 : 1;
  TRY_CUDA(dalloc(&p->d3, (size_t)p->elem * nfield * p->nmaps * kD3Tile * d3_tiles(p->npix), B));
  TRY_CUDA(dalloc(&p->alpha, (size_t)p->elem * 2 * p->npix, B));
  if (precision != TL_FP64) {
    TRY_CUDA(dalloc((void **)&p->gq, sizeof(int) * (size_t)p->npix, B));
    TRY_CUDA(dalloc((void **)&p->gq_count, sizeof(int), B));
  }
  TRY_CUDA(cudaDeviceSynchronize());

  const char *fb = getenv("TAYLENS_FFT_BATCH");
  p->fft_batch = fb ? atoi(fb) : 0;
  const char *env = getenv("TAYLENS_TIMING");
  p->timing = (env && env[0] == '1') ? 1 : 0;
  if (p->timing)
    for (int i = 0; i < 8; ++i) TRY_CUDA(cudaEventCreate(&p->ev[i]));
  if (p->timing)
    for (int i = 0; i < 3 * TL_MAX_BATCH; ++i) TRY_CUDA(cudaEventCreate(&p->evr[i]));
  return TL_OK;
}

extern "C" tl_status tl_plan_create(int nside, int lmax, int order, int spins, int precision, int flags,
                                    tl_plan **out) {
  if (!out) return TL_ERR_ARG;
  if (nside < 1 || nside > 8192 || (nside & (nside - 1)) != 0) return TL_ERR_ARG;
  if (lmax < 1 || lmax > 8 * nside) return TL_ERR_ARG;  // 8 nside: the paper's gradient band limit
  if (order < 0 || order > TL_MAX_ORDER) return TL_ERR_ARG;
  if (spins != TL_SPIN_T && spins != (TL_SPIN_T | TL_SPIN_QU)) {
    return (spins == TL_SPIN_QU) ? TL_ERR_UNSUPPORTED : TL_ERR_ARG;
  }
  if (precision < TL_FP64 || precision > TL_MIXED_BF16x3) return TL_ERR_ARG;
  if (flags & ~(TL_ROTATE | TL_NAIVE | TL_EXPAND_AT_PIXEL)) return TL_ERR_ARG;
  // the ring FFT keeps a whole ring in shared memory
  {
    tl_plan probe;
    memset(&probe, 0, sizeof(probe));
    probe.nside = nside;
    probe.precision = precision;
    int maxm = 0;
    for (int i = 1; i < nside; ++i) {
      if ((i & (i - 1)) == 0) continue;
      int M = 1;
      while (M < 2 * i - 1) M <<= 1;
      if (M > maxm) maxm = M;
    }
    probe.blue_maxm = maxm;  // as host_bluestein_layout, without its tables
    if (ringfft_smem_bytes(&probe) > 227 * 1024) return TL_ERR_UNSUPPORTED;
  }
  tl_plan *p = (tl_plan *)calloc(1, sizeof(tl_plan));
  if (!p) return TL_ERR_NOMEM;
  tl_status st = create_impl(nside, lmax, order, spins, precision, flags, p);
  if (st != TL_OK) {
    cudaDeviceSynchronize();
    free_plan(p);
    return st;
  }
  *out = p;
  return TL_OK;
}

extern "C" tl_status tl_plan_destroy(tl_plan *p) {
  if (!p) return TL_OK;
  cudaDeviceSynchronize();
  free_plan(p);
  return TL_OK;
}

extern "C" size_t tl_plan_workspace_bytes(const tl_plan *p) {
  return p ? p->bytes + (p->phi_plan ? p->phi_plan->bytes : 0) : 0;
}

extern "C" tl_status tl_plan_device_error(tl_plan *p) {
  if (!p) return TL_ERR_ARG;
  int h = 0;
  TRY_CUDA(cudaDeviceSynchronize());
  TRY_CUDA(cudaMemcpy(&h, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    TRY_CUDA(cudaMemset(p->dev_err, 0, sizeof(int)));
    return TL_ERR_TIMEOUT;
  }
  return TL_OK;
}

extern "C" tl_status tl_plan_set_wait_limit(tl_plan *p, int polls, int stall) {
  if (!p || polls < 0 || (stall != 0 && stall != 1)) return TL_ERR_ARG;
  p->wait_polls = polls;
  p->wait_stall = stall;
  return TL_OK;
}

extern "C" int tl_plan_maps_per_field(const tl_plan *p) { return p ? p->nmaps : 0; }
extern "C" int tl_plan_batch(const tl_plan *p) { return p ? p->batch : 0; }

extern "C" long long tl_plan_batch_launches(const tl_plan *p, int nreal, int with_phi) {
  if (!p || nreal < 0) return -1;
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  const long long G = p->fft_ngroups;  // one ring-FFT launch per ring group
  // a potential with its own band limit: prep, Legendre and FFT on its plan per realisation
  const long long sub = (with_phi && p->phi_plan) ? 2 + p->phi_plan->fft_ngroups : 0;
  const bool phi = with_phi != 0 && !p->phi_plan;
  if (p->batch > 1) {
    // per batch: coefficient tiles and Legendre launch of T, the potential and Q/U
    const long long chunks = (nreal + p->batch - 1) / p->batch;
    const long long per_chunk = 2 + (phi ? 2 : 0) + (pol ? 2 : 0);
    // per realisation: deflection FFT, derivative-map FFT, gather and its double pass
    return chunks * per_chunk + (long long)nreal * ((phi ? G : 0) + G + 2 + sub);
  }
  const bool fuse = phi && p->order >= 1;
  long long per = 0;
  if (phi && !fuse) per += 2 + G;  // stand-alone deflection: prep, Legendre, FFT
  per += 2 + (fuse ? 1 : 0);       // spin-0 prep (T, and phi when fused), Legendre
  if (fuse) per += G;              // deflection FFT
  if (pol) per += 2;               // spin-2 prep, Legendre
  per += G + (p->precision == TL_FP64 ? 1 : 2);  // derivative-map FFT, gather (float: and its double pass)
  return (long long)nreal * (per + sub);
}

// ---------------------------------------------------------------------------
// stages

static void mark(tl_plan *p, int i, cudaStream_t s) {
  if (p->timing && i < 8) cudaEventRecord(p->ev[i], s);
}

// alpha from the phi planes (j = 0, 1) already in d7_P
// il: the phi planes come from the tensor-core stage (four-ring interleaved rows)
static tl_status deflection_fft(tl_plan *p, void *ath, void *aph, cudaStream_t s, int il = 0) {
  const double L = deriv_norm(p);
  MapJob jobs[2] = {{3, 1, 0, 0, L, ath, 0, il}, {3, 0, 1, 1, L, aph, 0, il}};
  TRY_CUDA(launch_ringfft(p, jobs, 2, 2, s));
  return TL_OK;
}

// stand-alone deflection: phi through the spin-0 stage alone (uses rec_T)
static tl_status deflection_impl(tl_plan *p, const double *alm_phi, void *ath, void *aph, cudaStream_t s) {
  TRY_CUDA(launch_prep_spin0(p, alm_phi, nullptr, s));
  TRY_CUDA(launch_legendre_spin0(p, 1, false, p->d7_P, nullptr, s));
  return deflection_fft(p, ath, aph, s);
}

// the plan's deflection: on its own plan at lmax_phi when one is set
static tl_status plan_deflection(tl_plan *p, const double *alm_phi, void *ath, void *aph, cudaStream_t s) {
  return deflection_impl(p->phi_plan ? p->phi_plan : p, alm_phi, ath, aph, s);
}

extern "C" tl_status tl_deflection(tl_plan *p, const double *alm_phi, void *ath, void *aph, void *stream) {
  if (!p || !alm_phi || !ath || !aph) return TL_ERR_ARG;
  if (!aligned16(alm_phi) || !aligned16(ath) || !aligned16(aph)) return TL_ERR_ARG;
  return plan_deflection(p, alm_phi, ath, aph, (cudaStream_t)stream);
}

// Sec. II.A: the gradient of the potential is taken to its own band limit
// (min(8 Nside, 10000) in the paper). A separate deflection plan at lmax_phi (order
// 1, temperature only; single-precision SIMT form for the mixed forms, FP64 for FP64)
// then supplies alpha; lmax_phi = lmax removes it.
extern "C" tl_status tl_plan_set_lmax_phi(tl_plan *p, int lmax_phi) {
  if (!p || lmax_phi < 1) return TL_ERR_ARG;
  if (lmax_phi == p->lmax_phi) return TL_OK;
  TRY_CUDA(cudaDeviceSynchronize());  // queued work may still read the old plan or the staging
  if (p->phi_plan) {
    free_plan(p->phi_plan);
    p->phi_plan = nullptr;
  }
  // host-call staging is laid out for the potential's coefficient count
  const size_t slot_old = 3 * (size_t)nalm(p->lmax) * 16 + (size_t)nalm(p->lmax_phi) * 16;
  if (p->stage_alm) {
    cudaFree(p->stage_alm);
    p->bytes -= slot_old * (size_t)p->stage_cap;
    p->stage_alm = nullptr;
  }
  if (p->stage_out) {
    cudaFree(p->stage_out);
    p->bytes -= 3 * (size_t)p->elem * (size_t)p->npix * (size_t)p->stage_cap;
    p->stage_out = nullptr;
  }
  p->stage_cap = 0;
  p->lmax_phi = p->lmax;
  if (lmax_phi == p->lmax) return TL_OK;
  tl_plan *q = nullptr;
  const int prec = p->precision == TL_FP64 ? TL_FP64 : TL_MIXED_FP32;
  tl_status st = tl_plan_create(p->nside, lmax_phi, 1, TL_SPIN_T, prec, 0, &q);
  if (st != TL_OK) return st;
  p->phi_plan = q;
  p->lmax_phi = lmax_phi;
  return TL_OK;
}

static double fact(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

// (j, k), j + k <= order, in the order the ring FFT pairs them (jobs 2i and 2i+1
// share a transform): pairs within each plane j first, the left-overs of odd
// planes paired with each other at the end
static std::vector<std::pair<int, int>> paired_order(int order) {
  std::vector<std::pair<int, int>> out, rest;
  for (int j = 0; j <= order; ++j) {
    const int nk = order - j + 1;
    for (int k = 0; k + 1 < nk; k += 2) {
      out.push_back({j, k});
      out.push_back({j, k + 1});
    }
    if (nk & 1) rest.push_back({j, nk - 1});
  }
  out.insert(out.end(), rest.begin(), rest.end());
  return out;
}

extern "C" tl_status tl_synth_derivs(tl_plan *p, const double *alm, int spin, void *maps, void *stream) {
  if (!p || !alm || !maps) return TL_ERR_ARG;
  if (!aligned16(alm) || !aligned16(maps)) return TL_ERR_ARG;
  if (spin != 0 && spin != 2) return TL_ERR_ARG;
  if (spin == 2 && !(p->spins & TL_SPIN_QU)) return TL_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const double L = deriv_norm(p);
  const long long na = nalm(p->lmax);
  std::vector<MapJob> jobs;
  char *base = (char *)maps;
  const size_t mapb = (size_t)p->elem * p->npix;
  if (spin == 0) {
    TRY_CUDA(launch_prep_spin0(p, alm, nullptr, s));
    TRY_CUDA(launch_legendre_spin0(p, p->order, false, p->d7_T, nullptr, s));
    for (const std::pair<int, int> &jk : paired_order(p->order)) {
      const int j = jk.first, k = jk.second, n = j + k;
      jobs.push_back(MapJob{0, j, k, 0, pow(L, n), base + mapb * (n * (n + 1) / 2 + j)});
    }
  } else {
    TRY_CUDA(launch_prep_spin2(p, alm, alm + 2 * na, s));
    TRY_CUDA(launch_legendre_spin2(p, p->order, s));
    // Q and U of the same (j, k) share one packed transform (similar magnitudes)
    for (int n = 0; n <= p->order; ++n)
      for (int j = 0; j <= n; ++j)
        for (int f = 0; f < 2; ++f) {
          int k = n - j;
          jobs.push_back(MapJob{1 + f, j, k, 0, pow(L, n),
                                base + mapb * (f * p->nmaps + n * (n + 1) / 2 + j)});
        }
  }
  TRY_CUDA(launch_ringfft(p, jobs.data(), (int)jobs.size(), p->order + 1, s));
  return TL_OK;
}

// ring FFTs into Taylor-ready maps d_th^j d_ph^k s / (j! k! L^(j+k)) for one realisation
static tl_status lens_fft(tl_plan *p, const void *const *planes, cudaStream_t s, int il) {
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  std::vector<MapJob> jobs;
  // Jobs are packed two per transform in list order. Q and U of the same (j, k)
  // pair (similar magnitudes) and come first, an even count; then the T maps, which
  // pair within one coefficient plane j (the fold reads the row once for both),
  // left-overs across planes, the last one alone when their count is odd.
  // outputs in the pixel-tiled layout of d3 (map g * nmaps + index of (j, k))
  const long long tile = (long long)(pol ? 3 : 1) * p->nmaps * kD3Tile;
  auto out = [&](int map) { return (void *)((char *)p->d3 + (size_t)p->elem * map * kD3Tile); };
  if (pol)
    for (int n = 0; n <= p->order; ++n)
      for (int j = 0; j <= n; ++j)
        for (int g = 1; g < 3; ++g) {
          int k = n - j;
          jobs.push_back(MapJob{g, j, k, 0, 1.0 / (fact(j) * fact(k)), out(g * p->nmaps + n * (n + 1) / 2 + j), tile,
                                il});
        }
  for (const std::pair<int, int> &jk : paired_order(p->order))
    jobs.push_back(MapJob{0, jk.first, jk.second, 0, 1.0 / (fact(jk.first) * fact(jk.second)),
                          out((jk.first + jk.second) * (jk.first + jk.second + 1) / 2 + jk.first), tile, il});
  TRY_CUDA(launch_ringfft_planes(p, planes, jobs.data(), (int)jobs.size(), s));
  return TL_OK;
}

namespace tl {
// After the tensor-core Legendre stage of nreal realisations: per realisation the
// deflection's and the fields' ring FFTs, then the gather into the outputs.
tl_status lens_stage_after_legendre(tl_plan *p, int nreal, bool phi, void *const *To, void *const *Qo,
                                    void *const *Uo, cudaStream_t s, const double *const *aP) {
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  const size_t mapb = (size_t)p->elem * p->npix;
  const size_t t2 = 2 * (size_t)p->elem;
  void *ath = p->alpha, *aph = (char *)p->alpha + mapb;
  p->nevr = 0;
  for (int r = 0; r < nreal; ++r) {
      const bool tm = p->timing && r < TL_MAX_BATCH;
      if (tm) cudaEventRecord(p->evr[3 * r], s);
      const size_t off = (size_t)r * p->d7_rstride * t2, offp = (size_t)r * p->d7p_rstride * t2;
      const void *planes[4] = {(char *)p->d7_T + off, pol ? (char *)p->d7_Q + off : nullptr,
                               pol ? (char *)p->d7_U + off : nullptr, (char *)p->d7_P + offp};
      if (phi) {
        const double L = deriv_norm(p);
        MapJob jobs[2] = {{3, 1, 0, 0, L, ath, 0, 1}, {3, 0, 1, 1, L, aph, 0, 1}};
        TRY_CUDA(launch_ringfft_planes(p, planes, jobs, 2, s));
      } else if (aP && aP[r] && p->phi_plan) {
        tl_status st = plan_deflection(p, aP[r], ath, aph, s);
        if (st != TL_OK) return st;
      } else {
        TRY_CUDA(cudaMemsetAsync(p->alpha, 0, 2 * mapb, s));
      }
      tl_status st = lens_fft(p, planes, s, 1);
      if (st != TL_OK) return st;
      if (tm) cudaEventRecord(p->evr[3 * r + 1], s);
      TRY_CUDA(launch_gather(p, p->alpha, p->d3, To[r], pol ? Qo[r] : nullptr, pol ? Uo[r] : nullptr, s));
      if (p->done_rec && r < TL_MAX_BATCH) TRY_CUDA(cudaEventRecord(p->done_ev[r], s));
      if (tm) {
        cudaEventRecord(p->evr[3 * r + 2], s);
        p->nevr = r + 1;
      }
    }
  return TL_OK;
}
}  // namespace tl

// Lens nreal <= p->batch realisations that share one Legendre launch.
static tl_status lens_chunk(tl_plan *p, int nreal, const double *const *aT, const double *const *aE,
                            const double *const *aB, const double *const *aP, void *const *To, void *const *Qo,
                            void *const *Uo, cudaStream_t s) {
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  const size_t mapb = (size_t)p->elem * p->npix;
  const size_t t2 = 2 * (size_t)p->elem;
  void *ath = p->alpha, *aph = (char *)p->alpha + mapb;
  // the potential runs through the plan's own Legendre stage unless it has its own
  // band limit (then its deflection plan supplies alpha per realisation)
  const bool phi = aP[0] != nullptr && !p->phi_plan;
  p->nstage = 0;
  mark(p, 0, s);
  if (p->batch > 1) {
    // ---- tensor-core Legendre stage for all realisations of the chunk
    // the temperature at all orders, then the lensing potential at j <= 1 (its own
    // launch), then Q/U; on the host path the potential's and E/B's coefficients may
    // still be arriving on the copy stream while the temperature's launch runs
    TRY_CUDA(launch_tcprep(p, 0, nreal, aT, nullptr, p->tc_blk0, p->tab0, p->tc_b0, s));
    mark(p, 1, s);
    TRY_CUDA(launch_legendre_spin0_tc(p, 0, nreal, p->d7_T, p->d7_rstride, s));
    // (the potential's coefficients are also read later, by its own deflection plan
    // when it has one)
    if (p->in_wait && aP[0] != nullptr) TRY_CUDA(cudaStreamWaitEvent(s, p->in_ev[1], 0));
    if (phi) {
      TRY_CUDA(launch_tcprep(p, 0, nreal, aP, nullptr, p->tc_blk0, p->tab0, p->tc_bp, s));
      TRY_CUDA(launch_legendre_spin0_tc(p, 1, nreal, p->d7_P, p->d7p_rstride, s));
    }
    mark(p, 2, s);
    mark(p, 3, s);
    if (pol && p->in_wait) TRY_CUDA(cudaStreamWaitEvent(s, p->in_ev[2], 0));
    if (pol) TRY_CUDA(launch_tcprep(p, 2, nreal, aE, aB, p->tc_blk2, p->tab2, p->tc_b2, s));
    mark(p, 4, s);
    if (pol) TRY_CUDA(launch_legendre_spin2_tc(p, p->tc_nder, nreal, p->d7_Q, p->d7_U, p->d7_rstride, s));
    mark(p, 5, s);
    {
      tl_status st = lens_stage_after_legendre(p, nreal, phi, To, Qo, Uo, s, aP);
      if (st != TL_OK) return st;
    }
    mark(p, 6, s);
    mark(p, 7, s);
    p->nstage = p->timing ? 7 : 0;
    return TL_OK;
  }
  // ---- one realisation on the SIMT Legendre stage
  const double *alm_T = aT[0], *alm_E = aE ? aE[0] : nullptr, *alm_B = aB ? aB[0] : nullptr;
  const double *alm_phi = aP[0];
  // 1. spin-0 Legendre stage: T with all derivative orders; the lensing potential
  //    shares its basis for j <= 1 (needs order >= 1, else it runs on its own)
  const bool fuse = alm_phi && p->order >= 1 && !p->phi_plan;
  if (alm_phi && !fuse) {
    tl_status st = plan_deflection(p, alm_phi, ath, aph, s);
    if (st != TL_OK) return st;
  }
  TRY_CUDA(launch_prep_spin0(p, alm_T, fuse ? alm_phi : nullptr, s));
  mark(p, 1, s);
  TRY_CUDA(launch_legendre_spin0(p, p->order, fuse, p->d7_T, p->d7_P, s));
  mark(p, 2, s);
  // 2. deflection alpha = grad phi at the pixel centres
  if (fuse) {
    tl_status st = deflection_fft(p, ath, aph, s);
    if (st != TL_OK) return st;
  } else if (!alm_phi) {
    TRY_CUDA(cudaMemsetAsync(p->alpha, 0, 2 * mapb, s));
  }
  mark(p, 3, s);
  // 3. spin-2 Legendre stage
  if (pol) TRY_CUDA(launch_prep_spin2(p, alm_E, alm_B, s));
  mark(p, 4, s);
  if (pol) TRY_CUDA(launch_legendre_spin2(p, p->order, s));
  mark(p, 5, s);
  // 4. ring FFTs
  const void *planes[4] = {p->d7_T, p->d7_Q, p->d7_U, p->d7_P};
  tl_status st = lens_fft(p, planes, s, 0);
  if (st != TL_OK) return st;
  mark(p, 6, s);
  // 5. gather + Taylor + rotate
  TRY_CUDA(launch_gather(p, p->alpha, p->d3, To[0], pol ? Qo[0] : nullptr, pol ? Uo[0] : nullptr, s));
  mark(p, 7, s);
  p->nstage = p->timing ? 7 : 0;
  return TL_OK;
}

extern "C" tl_status tl_lens_batch(tl_plan *p, int nreal, const double *const *alm_T, const double *const *alm_E,
                                   const double *const *alm_B, const double *const *alm_phi, void *const *T_out,
                                   void *const *Q_out, void *const *U_out, void *stream) {
  if (!p || nreal < 0 || (nreal > 0 && (!alm_T || !T_out))) return TL_ERR_ARG;
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  if (pol && nreal > 0 && (!alm_E || !Q_out || !U_out)) return TL_ERR_ARG;
  for (int r = 0; r < nreal; ++r) {
    if (!alm_T[r] || !T_out[r]) return TL_ERR_ARG;
    if (pol && (!alm_E[r] || !Q_out[r] || !U_out[r])) return TL_ERR_ARG;
    const bool hp = alm_phi && alm_phi[r];
    const bool hp0 = alm_phi && alm_phi[0];
    if (hp != hp0) return TL_ERR_ARG;  // all realisations lensed, or none
    const void *ptrs[] = {alm_T[r], pol ? alm_E[r] : nullptr, (pol && alm_B) ? alm_B[r] : nullptr,
                          alm_phi ? alm_phi[r] : nullptr, T_out[r], pol ? Q_out[r] : nullptr,
                          pol ? U_out[r] : nullptr};
    for (const void *q : ptrs)
      if (q && !aligned16(q)) return TL_ERR_ARG;
  }
  static const double *const kNull[2] = {nullptr, nullptr};
  for (int r0 = 0; r0 < nreal; r0 += p->batch) {
    const int n = (nreal - r0) < p->batch ? (nreal - r0) : p->batch;
    tl_status st = lens_chunk(p, n, alm_T + r0, pol ? alm_E + r0 : nullptr, (pol && alm_B) ? alm_B + r0 : nullptr,
                              alm_phi ? alm_phi + r0 : kNull, T_out + r0, pol ? Q_out + r0 : nullptr,
                              pol ? U_out + r0 : nullptr, (cudaStream_t)stream);
    if (st != TL_OK) return st;
  }
  return TL_OK;
}

extern "C" tl_status tl_lens(tl_plan *p, const double *alm_T, const double *alm_E, const double *alm_B,
                             const double *alm_phi, void *T_out, void *Q_out, void *U_out, void *stream) {
  if (!p || !alm_T || !T_out) return TL_ERR_ARG;
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  if (pol && (!alm_E || !Q_out || !U_out)) return TL_ERR_ARG;
  const double *aT[1] = {alm_T}, *aE[1] = {alm_E}, *aB[1] = {alm_B}, *aP[1] = {alm_phi};
  void *To[1] = {T_out}, *Qo[1] = {Q_out}, *Uo[1] = {U_out};
  return tl_lens_batch(p, 1, aT, aE, aB, aP, To, Qo, Uo, stream);
}

// ---------------------------------------------------------------------------
// adjoint (reverse mode) of tl_lens

// The forward lens of one realisation up to its gather: Taylor-ready maps in d3
// and the deflection in alpha.
static tl_status forward_derivs(tl_plan *p, const double *alm_T, const double *alm_E, const double *alm_B,
                                const double *alm_phi, cudaStream_t s) {
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  const size_t mapb = (size_t)p->elem * p->npix;
  void *ath = p->alpha, *aph = (char *)p->alpha + mapb;
  bool defl_done = false;
  if (p->batch > 1) {
    const double *aT[1] = {alm_T}, *aE[1] = {alm_E}, *aB[1] = {alm_B}, *aP[1] = {alm_phi};
    TRY_CUDA(launch_tcprep(p, 0, 1, aT, nullptr, p->tc_blk0, p->tab0, p->tc_b0, s));
    if (alm_phi) TRY_CUDA(launch_tcprep(p, 0, 1, aP, nullptr, p->tc_blk0, p->tab0, p->tc_bp, s));
    TRY_CUDA(launch_legendre_spin0_tc(p, 0, 1, p->d7_T, p->d7_rstride, s));
    if (alm_phi) TRY_CUDA(launch_legendre_spin0_tc(p, 1, 1, p->d7_P, p->d7p_rstride, s));
    if (pol) {
      TRY_CUDA(launch_tcprep(p, 2, 1, aE, aB, p->tc_blk2, p->tab2, p->tc_b2, s));
      TRY_CUDA(launch_legendre_spin2_tc(p, p->tc_nder, 1, p->d7_Q, p->d7_U, p->d7_rstride, s));
    }
  } else {
    const bool fuse = alm_phi && p->order >= 1;
    if (alm_phi && !fuse) {
      tl_status st = deflection_impl(p, alm_phi, ath, aph, s);
      if (st != TL_OK) return st;
      defl_done = true;
    }
    TRY_CUDA(launch_prep_spin0(p, alm_T, fuse ? alm_phi : nullptr, s));
    TRY_CUDA(launch_legendre_spin0(p, p->order, fuse, p->d7_T, p->d7_P, s));
    if (pol) {
      TRY_CUDA(launch_prep_spin2(p, alm_E, alm_B, s));
      TRY_CUDA(launch_legendre_spin2(p, p->order, s));
    }
  }
  // the tensor-core stage leaves its planes four-ring interleaved
  const int il = p->batch > 1 ? 1 : 0;
  if (alm_phi && !defl_done) {
    tl_status st = deflection_fft(p, ath, aph, s, il);
    if (st != TL_OK) return st;
  } else if (!alm_phi) {
    TRY_CUDA(cudaMemsetAsync(p->alpha, 0, 2 * mapb, s));
  }
  const void *planes[4] = {p->d7_T, p->d7_Q, p->d7_U, p->d7_P};
  return lens_fft(p, planes, s, il);
}

extern "C" tl_status tl_lens_adjoint(tl_plan *p, const double *alm_T, const double *alm_E, const double *alm_B,
                                     const double *alm_phi, const void *gT, const void *gQ, const void *gU,
                                     double *galm_T, double *galm_E, double *galm_B, double *galm_phi, void *galpha,
                                     void *stream) {
  if (p && p->phi_plan) return TL_ERR_UNSUPPORTED;  // the potential's own band limit: forward only
  if (!p || !alm_T || !gT) return TL_ERR_ARG;
  if (p->flags & ~TL_ROTATE) return TL_ERR_UNSUPPORTED;  // the transpose of the default geometry only
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  if (pol && (!alm_E || !gQ || !gU)) return TL_ERR_ARG;
  if (!pol && (galm_E || galm_B)) return TL_ERR_ARG;
  const void *ptrs[] = {alm_T, alm_E, alm_B, alm_phi, gT, gQ, gU, galm_T, galm_E, galm_B, galm_phi, galpha};
  for (const void *q : ptrs)
    if (q && !aligned16(q)) return TL_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long long na = nalm(p->lmax);
  const size_t mapb = (size_t)p->elem * p->npix;
  const int nfield = pol ? 3 : 1;
  const size_t dbar_bytes = mapb * nfield * p->nmaps;
  if (!p->adj_dbar) TRY_CUDA(dalloc(&p->adj_dbar, dbar_bytes, &p->bytes));
  if (!galpha && !p->adj_ga) TRY_CUDA(dalloc(&p->adj_ga, 2 * mapb, &p->bytes));
  void *ga = galpha ? galpha : p->adj_ga;

  // stage marks (TAYLENS_TIMING): forward, gather, ring FFT, Legendre spin 0, spin 2, finish
  p->nstage = 0;
  mark(p, 0, s);
  // 1. forward quantities: d3 (Taylor-ready maps) and alpha
  {
    tl_status st = forward_derivs(p, alm_T, pol ? alm_E : nullptr, pol ? alm_B : nullptr, alm_phi, s);
    if (st != TL_OK) return st;
  }
  mark(p, 1, s);
  // 2. gather + Taylor + rotate, transposed: Dbar and the deflection gradient
  TRY_CUDA(cudaMemsetAsync(p->adj_dbar, 0, dbar_bytes, s));
  TRY_CUDA(launch_gather_adjoint(p, p->alpha, p->d3, gT, pol ? gQ : nullptr, pol ? gU : nullptr, p->adj_dbar, ga, s));
  mark(p, 2, s);
  // 3. ring synthesis, transposed, into the (now free) Legendre planes
  std::vector<AdjMapJob> jobs;
  const int n = p->order;
  for (int f = 0; f < nfield; ++f) {
    if (f == 0 && !galm_T) continue;
    if (f > 0 && !galm_E && !galm_B) continue;
    for (int j = 0; j <= n; ++j)
      jobs.push_back(AdjMapJob{f, j, n - j + 1, (const char *)p->adj_dbar + mapb * (size_t)f * p->nmaps});
  }
  if (galm_phi) {
    jobs.push_back(AdjMapJob{3, 1, 1, ga});
    jobs.push_back(AdjMapJob{3, 0, 1, (const char *)ga + mapb});
  }
  void *planes[4] = {p->d7_T, p->d7_Q, p->d7_U, p->d7_P};
  TRY_CUDA(launch_ringfft_adjoint(p, planes, jobs.data(), (int)jobs.size(), s));
  mark(p, 3, s);
  // 4. Legendre stages, transposed, accumulated straight into the outputs
  const size_t ab = (size_t)na * 16;
  double *outs[4] = {galm_T, galm_E, galm_B, galm_phi};
  for (double *o : outs)
    if (o) TRY_CUDA(cudaMemsetAsync(o, 0, ab, s));
  if (galm_T || galm_phi)
    TRY_CUDA(launch_legendre_adj0(p, galm_T ? n : -1, galm_T ? p->d7_T : nullptr, galm_phi ? p->d7_P : nullptr,
                                  galm_T, galm_phi, s));
  mark(p, 4, s);
  if (pol && (galm_E || galm_B)) {
    // A_{l+1} and m s/(l(l+1)) of the spin-2 step (prepared by the SIMT forward; the
    // tensor-core forward does not use these records)
    if (p->batch > 1) TRY_CUDA(launch_prep_spin2(p, alm_E, alm_B, s));
    TRY_CUDA(launch_legendre_adj2(p, n, p->d7_Q, p->d7_U, galm_E, galm_B, s));
  }
  mark(p, 5, s);
  TRY_CUDA(launch_adj_finish(p, galm_T, galm_phi, galm_E, galm_B, s));
  mark(p, 6, s);
  p->nstage = p->timing ? 6 : 0;
  return TL_OK;
}

extern "C" tl_status tl_lens_batch_host(tl_plan *p, int nreal, const double *const *alm_T,
                                        const double *const *alm_E, const double *const *alm_B,
                                        const double *const *alm_phi, void *const *T_out, void *const *Q_out,
                                        void *const *U_out, void *stream) {
  if (!p || nreal < 0 || (nreal > 0 && (!alm_T || !T_out))) return TL_ERR_ARG;
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  if (pol && nreal > 0 && (!alm_E || !Q_out || !U_out)) return TL_ERR_ARG;
  for (int r = 0; r < nreal; ++r) {
    if (!alm_T[r] || !T_out[r]) return TL_ERR_ARG;
    if (pol && (!alm_E[r] || !Q_out[r] || !U_out[r])) return TL_ERR_ARG;
    if ((alm_phi && alm_phi[r]) != (alm_phi && alm_phi[0])) return TL_ERR_ARG;  // all lensed, or none
  }
  if (nreal == 0) return TL_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const long long na = nalm(p->lmax);
  const size_t ab = (size_t)na * 16, mapb = (size_t)p->elem * p->npix;
  const size_t abp = (size_t)nalm(p->lmax_phi) * 16;  // the potential's coefficients
  const size_t slot = 3 * ab + abp;                    // staging per realisation
  // device staging for one chunk of up to p->batch realisations (one Legendre launch
  // on tensor-core plans), grown on demand and kept by the plan
  const int cap = nreal < p->batch ? nreal : p->batch;
  if (cap > p->stage_cap) {
    if (p->stage_alm || p->stage_out) TRY_CUDA(cudaStreamSynchronize(s));
    if (p->stage_alm) {
      cudaFree(p->stage_alm);
      p->bytes -= slot * (size_t)p->stage_cap;
      p->stage_alm = nullptr;
    }
    if (p->stage_out) {
      cudaFree(p->stage_out);
      p->bytes -= 3 * mapb * (size_t)p->stage_cap;
      p->stage_out = nullptr;
    }
    p->stage_cap = 0;
    TRY_CUDA(dalloc(&p->stage_alm, slot * (size_t)cap, &p->bytes));
    TRY_CUDA(dalloc(&p->stage_out, 3 * mapb * (size_t)cap, &p->bytes));
    p->stage_cap = cap;
  }
  const bool phi = alm_phi && alm_phi[0];
  for (int r0 = 0; r0 < nreal; r0 += cap) {
    const int n = (nreal - r0) < cap ? (nreal - r0) : cap;
    const double *dT[TL_MAX_BATCH], *dE[TL_MAX_BATCH], *dB[TL_MAX_BATCH], *dP[TL_MAX_BATCH];
    void *oT[TL_MAX_BATCH], *oQ[TL_MAX_BATCH], *oU[TL_MAX_BATCH];
    for (int i = 0; i < n; ++i) {
      const int r = r0 + i;
      char *a = (char *)p->stage_alm + slot * (size_t)i;
      char *o = (char *)p->stage_out + 3 * mapb * (size_t)i;
      dT[i] = (const double *)a;
      dE[i] = pol ? (const double *)(a + ab) : nullptr;
      dB[i] = (pol && alm_B && alm_B[r]) ? (const double *)(a + 2 * ab) : nullptr;
      dP[i] = phi ? (const double *)(a + 3 * ab) : nullptr;
      oT[i] = o;
      oQ[i] = pol ? o + mapb : nullptr;
      oU[i] = pol ? o + 2 * mapb : nullptr;
    }
    // On tensor-core plans a chunk's realisations run their ring FFTs and gathers one
    // after another, so each one's maps are copied back on a second stream as soon as its
    // gather has run, while the later ones are still being computed; and only the
    // temperature's coefficients are needed before the first Legendre launch, so the
    // potential's and E/B's arrive on that stream meanwhile.
    const bool overlap = p->batch > 1 && n > 1;
    if (overlap && !p->copy_stream) {
      TRY_CUDA(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
      for (int i = 0; i < TL_MAX_BATCH; ++i) TRY_CUDA(cudaEventCreateWithFlags(&p->done_ev[i], cudaEventDisableTiming));
      TRY_CUDA(cudaEventCreateWithFlags(&p->copied_ev, cudaEventDisableTiming));
      for (int i = 0; i < 3; ++i) TRY_CUDA(cudaEventCreateWithFlags(&p->in_ev[i], cudaEventDisableTiming));
    }
    cudaStream_t ins = overlap ? p->copy_stream : s;
    for (int i = 0; i < n; ++i)
      TRY_CUDA(cudaMemcpyAsync((void *)dT[i], alm_T[(size_t)r0 + i], ab, cudaMemcpyHostToDevice, s));
    if (overlap) {
      // the staging is free once the compute stream has passed the previous chunk
      TRY_CUDA(cudaEventRecord(p->in_ev[0], s));
      TRY_CUDA(cudaStreamWaitEvent(ins, p->in_ev[0], 0));
    }
    for (int i = 0; i < n; ++i)
      if (dP[i]) TRY_CUDA(cudaMemcpyAsync((void *)dP[i], alm_phi[(size_t)r0 + i], abp, cudaMemcpyHostToDevice, ins));
    if (overlap) TRY_CUDA(cudaEventRecord(p->in_ev[1], ins));
    for (int i = 0; i < n; ++i) {
      if (dE[i]) TRY_CUDA(cudaMemcpyAsync((void *)dE[i], alm_E[(size_t)r0 + i], ab, cudaMemcpyHostToDevice, ins));
      if (dB[i]) TRY_CUDA(cudaMemcpyAsync((void *)dB[i], alm_B[(size_t)r0 + i], ab, cudaMemcpyHostToDevice, ins));
    }
    if (overlap) TRY_CUDA(cudaEventRecord(p->in_ev[2], ins));
    if (overlap) {
      // the previous chunk's copies read the staging this chunk overwrites
      TRY_CUDA(cudaStreamWaitEvent(s, p->copied_ev, 0));
    }
    p->done_rec = overlap ? 1 : 0;
    p->in_wait = overlap ? 1 : 0;
    tl_status st = tl_lens_batch(p, n, dT, pol ? dE : nullptr, pol ? dB : nullptr, dP, oT, pol ? oQ : nullptr,
                                 pol ? oU : nullptr, stream);
    p->done_rec = 0;
    p->in_wait = 0;
    if (st != TL_OK) return st;
    cudaStream_t cs = overlap ? p->copy_stream : s;
    for (int i = 0; i < n; ++i) {
      const int r = r0 + i;
      if (overlap) TRY_CUDA(cudaStreamWaitEvent(cs, p->done_ev[i], 0));
      TRY_CUDA(cudaMemcpyAsync(T_out[r], oT[i], mapb, cudaMemcpyDeviceToHost, cs));
      if (pol) {
        TRY_CUDA(cudaMemcpyAsync(Q_out[r], oQ[i], mapb, cudaMemcpyDeviceToHost, cs));
        TRY_CUDA(cudaMemcpyAsync(U_out[r], oU[i], mapb, cudaMemcpyDeviceToHost, cs));
      }
    }
    if (overlap) TRY_CUDA(cudaEventRecord(p->copied_ev, cs));
  }
  TRY_CUDA(cudaStreamSynchronize(s));
  if (p->copy_stream) TRY_CUDA(cudaStreamSynchronize(p->copy_stream));
  return TL_OK;
}

extern "C" tl_status tl_lens_host(tl_plan *p, const double *alm_T, const double *alm_E, const double *alm_B,
                                  const double *alm_phi, void *T_out, void *Q_out, void *U_out, void *stream) {
  if (!p || !alm_T || !T_out) return TL_ERR_ARG;
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  if (pol && (!alm_E || !Q_out || !U_out)) return TL_ERR_ARG;
  const double *aT[1] = {alm_T}, *aE[1] = {alm_E}, *aB[1] = {alm_B}, *aP[1] = {alm_phi};
  void *To[1] = {T_out}, *Qo[1] = {Q_out}, *Uo[1] = {U_out};
  return tl_lens_batch_host(p, 1, aT, aE, aB, aP, To, Qo, Uo, stream);
}

extern "C" int tl_last_stage_ms(const tl_plan *p, float *ms, int n) {
  if (!p || !ms || !p->timing || p->nstage == 0) return 0;
  tl_plan *q = (tl_plan *)p;
  if (cudaEventSynchronize(q->ev[p->nstage]) != cudaSuccess) return 0;
  int k = 0;
  for (int i = 0; i < p->nstage && k < n; ++i, ++k) cudaEventElapsedTime(&ms[k], q->ev[i], q->ev[i + 1]);
  if (p->nstage == 7 && k + 2 <= n) {
    // ring FFTs and gathers of the call
    float fft = 0.f, gat = 0.f;
    if (p->batch > 1) {
      for (int r = 0; r < p->nevr; ++r) {
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, q->evr[3 * r], q->evr[3 * r + 1]);
        cudaEventElapsedTime(&b, q->evr[3 * r + 1], q->evr[3 * r + 2]);
        fft += a;
        gat += b;
      }
    } else {
      fft = ms[2] + ms[5];
      gat = ms[6];
    }
    ms[k++] = fft;
    ms[k++] = gat;
  }
  return k;
}
