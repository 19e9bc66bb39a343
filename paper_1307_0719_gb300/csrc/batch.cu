// Batched lensing of many realisations of uneven size (tl_batch_*).
//
// Realisations are grouped by geometry (nside, lmax); each group owns a plan.
// On tensor-core plans the work goes in waves: a wave takes the next realisations,
// up to the plan's batch (16 at orders up to 5, 8 above), from every group that
// still has some, prepares their coefficient
// fragments, and runs the Legendre stage of all of them in ONE persistent
// launch whose blocks pull (plan, spin, m, ring block) items, pre-sorted by cost,
// from an atomic counter; ring FFTs and the gather then follow per realisation.
// The whole sequence can be captured once in a CUDA graph and replayed. The
// reference point is a plain per-realisation loop of tl_lens calls. An autotuner
// times the persistent grid size and the ring-FFT batching on the caller's data
// and keeps the choice (optionally in a cache file named by TAYLENS_TUNE_CACHE).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "legendre.cuh"

namespace tl {
void tc_desc_write(const tl_plan *p, int which, int nreal, void *dst);
size_t tc_desc_bytes();
cudaError_t launch_legendre_tc_persistent(int nder, int precision, const void *descs, const void *items, int nitems,
                                          int *counter, int grid, cudaStream_t s);
tl_status lens_stage_after_legendre(tl_plan *p, int nreal, bool phi, void *const *To, void *const *Qo,
                                    void *const *Uo, cudaStream_t s,
                                    const double *const *aP);
}  // namespace tl

using namespace tl;

struct Wave {
  std::vector<std::pair<int, int>> members;  // (group, first realisation index within the group's list)
  std::vector<int> counts;                   // realisations of each member in this wave (1 or 2)
  long long item_off;                        // into the device item array
  int nitems;
  long long desc_off;                        // into the device descriptor array (3 per member)
};

struct tl_batch {
  int nreal, order, spins, precision, flags;
  std::vector<tl_plan *> plans;              // one per group
  std::vector<int> group_of;                 // realisation -> group
  std::vector<std::vector<int>> members;     // group -> realisations
  std::vector<Wave> waves;
  bool persistent_ok;
  void *d_items, *d_descs;
  int *d_counter;                            // one counter per wave
  int grid;                                  // persistent grid size
  // graph
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  std::vector<const void *> graph_ptrs;      // pointers the graph was captured with
  cudaStream_t graph_stream;
};

static tl_status st_cuda(cudaError_t e) {
  return e == cudaSuccess ? TL_OK : (e == cudaErrorMemoryAllocation ? TL_ERR_NOMEM : TL_ERR_CUDA);
}
#define B_TRY(call)                        \
  do {                                     \
    cudaError_t _e = (call);               \
    if (_e != cudaSuccess) return st_cuda(_e); \
  } while (0)

static void batch_free(tl_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (tl_plan *p : b->plans) tl_plan_destroy(p);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_descs) cudaFree(b->d_descs);
  if (b->d_counter) cudaFree(b->d_counter);
  delete b;
}

static std::string tune_key(const tl_batch *b) {
  char buf[256];
  std::string k;
  snprintf(buf, sizeof buf, "o%d_s%d_p%d", b->order, b->spins, b->precision);
  k = buf;
  for (size_t g = 0; g < b->plans.size(); ++g) {
    snprintf(buf, sizeof buf, "_%dx%d:%d", b->plans[g]->nside, b->plans[g]->lmax, (int)b->members[g].size());
    k += buf;
  }
  return k;
}

// cache lines: "<key> <grid> <fft_batch of group 0> <fft_batch of group 1> ..."
static bool tune_load(tl_batch *b) {
  const char *path = getenv("TAYLENS_TUNE_CACHE");
  if (!path) return false;
  FILE *f = fopen(path, "r");
  if (!f) return false;
  const std::string key = tune_key(b);
  char line[4096];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char k[2048];
    int n = 0;
    if (sscanf(line, "%2047s%n", k, &n) != 1 || key != k) continue;
    const char *q = line + n;
    int grid, used;
    if (sscanf(q, "%d%n", &grid, &used) != 1) continue;
    q += used;
    std::vector<int> fb;
    int v;
    while (sscanf(q, "%d%n", &v, &used) == 1) {
      fb.push_back(v);
      q += used;
    }
    if (fb.size() != b->plans.size()) continue;
    b->grid = grid;
    for (size_t g = 0; g < fb.size(); ++g) b->plans[g]->fft_batch = fb[g];
    found = true;
  }
  fclose(f);
  return found;
}

static void tune_store(const tl_batch *b) {
  const char *path = getenv("TAYLENS_TUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d", tune_key(b).c_str(), b->grid);
  for (tl_plan *p : b->plans) fprintf(f, " %d", p->fft_batch);
  fprintf(f, "\n");
  fclose(f);
}

extern "C" tl_status tl_batch_create(int nreal, const int *nside, const int *lmax, int order, int spins,
                                     int precision, int flags, tl_batch **out) {
  if (!out || nreal < 1 || !nside || !lmax) return TL_ERR_ARG;
  tl_batch *b = new (std::nothrow) tl_batch();
  if (!b) return TL_ERR_NOMEM;
  b->nreal = nreal;
  b->order = order;
  b->spins = spins;
  b->precision = precision;
  b->flags = flags;
  b->grid = 0;
  std::map<std::pair<int, int>, int> gid;
  b->group_of.resize(nreal);
  for (int i = 0; i < nreal; ++i) {
    auto key = std::make_pair(nside[i], lmax[i]);
    auto it = gid.find(key);
    int g;
    if (it == gid.end()) {
      tl_plan *p = nullptr;
      tl_status st = tl_plan_create(nside[i], lmax[i], order, spins, precision, flags, &p);
      if (st != TL_OK) {
        batch_free(b);
        return st;
      }
      g = (int)b->plans.size();
      gid[key] = g;
      b->plans.push_back(p);
      b->members.emplace_back();
    } else {
      g = it->second;
    }
    b->group_of[i] = g;
    b->members[g].push_back(i);
  }
  b->persistent_ok = b->plans[0]->batch > 1;
  if (b->persistent_ok) {
    // waves and their cost-sorted item lists; descriptors (temperature, potential,
    // polarisation) per member
    const size_t db = tc_desc_bytes();
    std::vector<int4> items;
    std::vector<unsigned char> descs;
    std::vector<const tl_plan *> desc_plan;  // geometry behind each descriptor (for the checks below)
    size_t maxc = 0;
    const size_t per = (size_t)b->plans[0]->batch;  // realisations per wave and group
    for (auto &m : b->members) maxc = std::max(maxc, (m.size() + per - 1) / per);
    const bool pol = (spins & TL_SPIN_QU) != 0;
    for (size_t w = 0; w < maxc; ++w) {
      Wave wv;
      wv.item_off = (long long)items.size();
      wv.desc_off = (long long)(descs.size() / db);
      struct It {
        long long cost;
        int4 v;
      };
      std::vector<It> its;
      for (size_t g = 0; g < b->plans.size(); ++g) {
        const size_t first = per * w;
        if (first >= b->members[g].size()) continue;
        const int cnt = (int)std::min<size_t>(per, b->members[g].size() - first);
        const int di = (int)(descs.size() / db);
        for (int which : {0, 1, 2}) {
          const size_t at = descs.size();
          descs.resize(at + db);
          tc_desc_write(b->plans[g], which, cnt, descs.data() + at);
          desc_plan.push_back(b->plans[g]);
        }
        wv.members.push_back(std::make_pair((int)g, (int)first));
        wv.counts.push_back(cnt);
        const tl_plan *p = b->plans[g];
        const int nb0 = tc_ring_blocks(p, 0), nb2 = tc_ring_blocks(p, 2);
        // cost ~ blocks x (recurrence + tiles of NDER + 1 orders); the potential carries 2
        const long long wt = p->tc_nder + 1, wp = 2;
        for (int m = 0; m <= p->mmax; ++m) {
          for (int r = 0; r < nb0; ++r) {
            its.push_back({(long long)(p->lmax - m + 1) * wt, make_int4(di | (0 << 16), m, r, 0)});
            its.push_back({(long long)(p->lmax - m + 1) * wp, make_int4((di + 1) | (1 << 16), m, r, 0)});
          }
          if (pol)
            for (int r = 0; r < nb2; ++r)
              its.push_back({(long long)(p->lmax - std::max(m, 2) + 1) * wt, make_int4((di + 2) | (2 << 16), m, r, 0)});
        }
      }
      std::stable_sort(its.begin(), its.end(), [](const It &x, const It &y) { return x.cost > y.cost; });
      for (auto &x : its) items.push_back(x.v);
      wv.nitems = (int)its.size();
      b->waves.push_back(wv);
    }
    // every item must name an existing descriptor, an m of its plan and a ring block inside its rings
    for (const int4 &v : items) {
      const int di = v.x & 0xffff, kind = v.x >> 16;
      if (di < 0 || di >= (int)desc_plan.size() || kind < 0 || kind > 2) {
        batch_free(b);
        return TL_ERR_ARG;
      }
      const tl_plan *q = desc_plan[di];
      const int nbk = tc_ring_blocks(q, kind == 2 ? 2 : 0);
      if (v.y < 0 || v.y > q->mmax || v.z < 0 || v.z >= nbk || di % 3 != kind) {
        batch_free(b);
        return TL_ERR_ARG;
      }
    }
    cudaError_t e = cudaMalloc(&b->d_items, sizeof(int4) * items.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_descs, descs.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->d_descs, descs.data(), descs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_counter, sizeof(int) * b->waves.size());
    if (e != cudaSuccess) {
      batch_free(b);
      return st_cuda(e);
    }
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    b->grid = nsm * tc_persistent_ctas(b->plans[0]->tc_nder, precision);  // as the tensor memory allows
  }
  tune_load(b);
  *out = b;
  return TL_OK;
}

extern "C" tl_status tl_batch_destroy(tl_batch *b) {
  if (!b) return TL_OK;
  cudaDeviceSynchronize();
  batch_free(b);
  return TL_OK;
}

extern "C" int tl_batch_groups(const tl_batch *b) { return b ? (int)b->plans.size() : 0; }
extern "C" int tl_batch_waves(const tl_batch *b) { return b ? (int)b->waves.size() : 0; }
extern "C" int tl_batch_grid(const tl_batch *b) { return b ? b->grid : 0; }

// one pass: per-realisation loop (mode 0) or waves with the persistent Legendre launch (mode 1)
static tl_status batch_pass(tl_batch *b, int mode, const double *const *aT, const double *const *aE,
                            const double *const *aB, const double *const *aP, void *const *To, void *const *Qo,
                            void *const *Uo, cudaStream_t s) {
  const bool pol = (b->spins & TL_SPIN_QU) != 0;
  const bool phi = aP && aP[0];
  if (mode == 0 || !b->persistent_ok) {
    for (int i = 0; i < b->nreal; ++i) {
      tl_plan *p = b->plans[b->group_of[i]];
      tl_status st = tl_lens(p, aT[i], pol ? aE[i] : nullptr, (pol && aB) ? aB[i] : nullptr, phi ? aP[i] : nullptr,
                             To[i], pol ? Qo[i] : nullptr, pol ? Uo[i] : nullptr, s);
      if (st != TL_OK) return st;
    }
    return TL_OK;
  }
  for (size_t w = 0; w < b->waves.size(); ++w) {
    const Wave &wv = b->waves[w];
    // coefficient tiles of every member group
    for (size_t k = 0; k < wv.members.size(); ++k) {
      const int g = wv.members[k].first, first = wv.members[k].second, cnt = wv.counts[k];
      tl_plan *p = b->plans[g];
      const double *t[TL_MAX_BATCH], *e[TL_MAX_BATCH], *bb[TL_MAX_BATCH], *ph[TL_MAX_BATCH];
      for (int r = 0; r < cnt; ++r) {
        const int i = b->members[g][first + r];
        t[r] = aT[i];
        e[r] = pol ? aE[i] : nullptr;
        bb[r] = (pol && aB) ? aB[i] : nullptr;
        ph[r] = phi ? aP[i] : nullptr;
      }
      B_TRY(launch_tcprep(p, 0, cnt, t, nullptr, p->tc_blk0, p->tab0, p->tc_b0, s));
      if (phi) B_TRY(launch_tcprep(p, 0, cnt, ph, nullptr, p->tc_blk0, p->tab0, p->tc_bp, s));
      if (pol) B_TRY(launch_tcprep(p, 2, cnt, e, bb, p->tc_blk2, p->tab2, p->tc_b2, s));
    }
    // the Legendre stage of the whole wave in one persistent launch
    const int4 *items = (const int4 *)b->d_items + wv.item_off;
    // items index the whole descriptor array (indices were assigned across all waves)
    const unsigned char *descs = (const unsigned char *)b->d_descs;
    B_TRY(cudaMemsetAsync(b->d_counter + w, 0, sizeof(int), s));
    B_TRY(launch_legendre_tc_persistent(b->plans[0]->tc_nder, b->precision, descs, items, wv.nitems,
                                        b->d_counter + w, b->grid, s));
    // ring FFTs and gather per realisation
    for (size_t k = 0; k < wv.members.size(); ++k) {
      const int g = wv.members[k].first, first = wv.members[k].second, cnt = wv.counts[k];
      void *T2[TL_MAX_BATCH], *Q2[TL_MAX_BATCH], *U2[TL_MAX_BATCH];
      for (int r = 0; r < cnt; ++r) {
        const int i = b->members[g][first + r];
        T2[r] = To[i];
        Q2[r] = pol ? Qo[i] : nullptr;
        U2[r] = pol ? Uo[i] : nullptr;
      }
      tl_status st = lens_stage_after_legendre(b->plans[g], cnt, phi, T2, Q2, U2, s, nullptr);
      if (st != TL_OK) return st;
    }
  }
  return TL_OK;
}

static bool same_ptrs(const tl_batch *b, const std::vector<const void *> &v) { return b->graph_ptrs == v; }

extern "C" tl_status tl_batch_lens(tl_batch *b, int mode, const double *const *alm_T, const double *const *alm_E,
                                   const double *const *alm_B, const double *const *alm_phi, void *const *T_out,
                                   void *const *Q_out, void *const *U_out, void *stream) {
  if (!b || !alm_T || !T_out || mode < 0 || mode > 2) return TL_ERR_ARG;
  const bool pol = (b->spins & TL_SPIN_QU) != 0;
  if (pol && (!alm_E || !Q_out || !U_out)) return TL_ERR_ARG;
  const bool phi = alm_phi && alm_phi[0];
  if (b->persistent_ok && mode > 0 && !phi) return TL_ERR_UNSUPPORTED;  // waves assume the potential is present
  for (int i = 0; i < b->nreal; ++i) {
    if (!alm_T[i] || !T_out[i] || (pol && (!alm_E[i] || !Q_out[i] || !U_out[i]))) return TL_ERR_ARG;
    if ((alm_phi && alm_phi[i]) != phi) return TL_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (mode < 2 || !b->persistent_ok)
    return batch_pass(b, mode > 0 ? 1 : 0, alm_T, alm_E, alm_B, alm_phi, T_out, Q_out, U_out, s);
  // mode 2: capture once per set of pointers, then replay
  std::vector<const void *> key;
  for (int i = 0; i < b->nreal; ++i) {
    key.push_back(alm_T[i]);
    key.push_back(pol ? alm_E[i] : nullptr);
    key.push_back((pol && alm_B) ? alm_B[i] : nullptr);
    key.push_back(phi ? alm_phi[i] : nullptr);
    key.push_back(T_out[i]);
    key.push_back(pol ? Q_out[i] : nullptr);
    key.push_back(pol ? U_out[i] : nullptr);
  }
  if (!b->exec || !same_ptrs(b, key)) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    if (b->graph) {
      cudaGraphDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaStream_t cs;
    B_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    tl_status st = TL_OK;
    if (e == cudaSuccess) {
      st = batch_pass(b, 1, alm_T, alm_E, alm_B, alm_phi, T_out, Q_out, U_out, cs);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(cs, &g);
      b->graph = g;
    }
    cudaStreamDestroy(cs);
    if (st != TL_OK) return st;
    B_TRY(e);
    B_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->graph_ptrs = key;
  }
  B_TRY(cudaGraphLaunch(b->exec, s));
  return TL_OK;
}

// Time candidate persistent grids and ring-FFT batching on the caller's data; keep
// the fastest (and append it to TAYLENS_TUNE_CACHE when set). Synchronises.
extern "C" tl_status tl_batch_autotune(tl_batch *b, const double *const *alm_T, const double *const *alm_E,
                                       const double *const *alm_B, const double *const *alm_phi,
                                       void *const *T_out, void *const *Q_out, void *const *U_out, void *stream) {
  if (!b) return TL_ERR_ARG;
  if (!b->persistent_ok || !(alm_phi && alm_phi[0])) return TL_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t e0, e1;
  B_TRY(cudaEventCreate(&e0));
  B_TRY(cudaEventCreate(&e1));
  auto timeit = [&](float *ms) -> tl_status {
    tl_status st = batch_pass(b, 1, alm_T, alm_E, alm_B, alm_phi, T_out, Q_out, U_out, s);  // warm
    if (st != TL_OK) return st;
    cudaEventRecord(e0, s);
    st = batch_pass(b, 1, alm_T, alm_E, alm_B, alm_phi, T_out, Q_out, U_out, s);
    cudaEventRecord(e1, s);
    if (st != TL_OK) return st;
    if (cudaEventSynchronize(e1) != cudaSuccess) return TL_ERR_CUDA;
    cudaEventElapsedTime(ms, e0, e1);
    return TL_OK;
  };
  // 1. ring-FFT batching (one knob per group, all groups together)
  float best = 1e30f;
  int best_fb = 1;
  for (int fb : {1, 4}) {
    for (tl_plan *p : b->plans) p->fft_batch = fb;
    float ms;
    tl_status st = timeit(&ms);
    if (st != TL_OK) return st;
    if (ms < best) {
      best = ms;
      best_fb = fb;
    }
  }
  for (tl_plan *p : b->plans) p->fft_batch = best_fb;
  // 2. persistent grid size (blocks per SM)
  best = 1e30f;
  int best_grid = b->grid;
  const int ctas = tc_persistent_ctas(b->plans[0]->tc_nder, b->precision);
  for (int k : {ctas > 1 ? ctas / 2 : 1, ctas}) {
    b->grid = nsm * k;
    float ms;
    tl_status st = timeit(&ms);
    if (st != TL_OK) return st;
    if (ms < best) {
      best = ms;
      best_grid = b->grid;
    }
  }
  b->grid = best_grid;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (b->exec) {  // settings changed: recapture on the next graph call
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_ptrs.clear();
  }
  tune_store(b);
  return TL_OK;
}
