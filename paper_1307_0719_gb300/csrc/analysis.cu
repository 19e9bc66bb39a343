// Analysis side of the lensed maps (Naess & Louis 2013, Sec. III: the paper
// measures its accuracy on angular power spectra of the lensed maps, from
// healpy's map2alm and anafast):
//   tl_map2alm: a_lm = (4 pi / Npix) sum_p s(p) conj(sY_lm(p)), uniform weights and
//     no iteration (healpy's default map2alm), spin 0 (T) and spin 2 (Q, U -> E, B
//     in the HEALPix convention of the synthesis). It is the transpose of the ring
//     synthesis with those weights, so it runs the adjoint kernels of tl_lens_adjoint
//     at order 0: the adjoint ring FFT of each map into the per-ring planes, the
//     transposed Legendre contraction and the k_l scaling, then the weights.
//   tl_anafast: C_l^XY = (1/(2l+1)) sum_m Re(a_lm conj(b_lm)), m = -l..l, for the
//     pairs TT, EE, BB, TE, TB, EB.
#include "common.cuh"

namespace tl {

// (4 pi / Npix) grad / w_m: the gradient of sum_p g s with respect to a real field's
// coefficient carries w_m = 2 for m > 0 (a_lm and a_l,-m = (-1)^m conj a_lm both)
__global__ void map2alm_weight_kernel(int lmax, double w, double *__restrict__ a) {
  const int m = blockIdx.y;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax || !a) return;
  const long long idx = (long long)m * (2 * lmax + 1 - m) / 2 + l;
  const double f = (m == 0) ? w : 0.5 * w;
  a[2 * idx] *= f;
  a[2 * idx + 1] *= f;
}

// One thread per l; sums over m in healpy order (idx = m (2 lmax + 1 - m) / 2 + l).
__global__ void anafast_kernel(int lmax, const double *__restrict__ aT, const double *__restrict__ aE,
                               const double *__restrict__ aB, double *__restrict__ cl) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  const double *f[3] = {aT, aE, aB};
  const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  for (int q = 0; q < 6; ++q) {
    const double *x = f[pairs[q][0]], *y = f[pairs[q][1]];
    if (!x || !y) continue;
    double s = 0.0;
    for (int m = 0; m <= l; ++m) {
      const long long idx = (long long)m * (2 * lmax + 1 - m) / 2 + l;
      const double v = x[2 * idx] * y[2 * idx] + x[2 * idx + 1] * y[2 * idx + 1];
      s += (m == 0) ? v : 2.0 * v;
    }
    cl[(size_t)q * (lmax + 1) + l] = s / (2.0 * l + 1.0);
  }
}

}  // namespace tl

using namespace tl;

static bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

extern "C" tl_status tl_map2alm(tl_plan *p, const void *T, const void *Q, const void *U, double *alm_T,
                                double *alm_E, double *alm_B, void *stream) {
  if (!p || !T || !alm_T) return TL_ERR_ARG;
  const bool pol = (p->spins & TL_SPIN_QU) != 0;
  const bool want_pol = Q || U || alm_E || alm_B;
  if (want_pol && (!pol || !Q || !U || !alm_E || !alm_B)) return TL_ERR_ARG;
  const void *ptrs[] = {T, Q, U, alm_T, alm_E, alm_B};
  for (const void *q : ptrs)
    if (q && !al16(q)) return TL_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ab = (size_t)nalm(p->lmax) * 16;
  AdjMapJob jobs[3];
  int nj = 0;
  jobs[nj++] = AdjMapJob{0, 0, 1, T};
  if (want_pol) {
    jobs[nj++] = AdjMapJob{1, 0, 1, Q};
    jobs[nj++] = AdjMapJob{2, 0, 1, U};
  }
  void *planes[4] = {p->d7_T, p->d7_Q, p->d7_U, p->d7_P};
  TL_CUDA_TRY_STATUS(launch_ringfft_adjoint(p, planes, jobs, nj, s));
  TL_CUDA_TRY_STATUS(cudaMemsetAsync(alm_T, 0, ab, s));
  TL_CUDA_TRY_STATUS(launch_legendre_adj0(p, 0, p->d7_T, nullptr, alm_T, nullptr, s));
  if (want_pol) {
    TL_CUDA_TRY_STATUS(cudaMemsetAsync(alm_E, 0, ab, s));
    TL_CUDA_TRY_STATUS(cudaMemsetAsync(alm_B, 0, ab, s));
    // step factors of the spin-2 recurrence (the coefficient fields of the records
    // are not read by the transposed contraction)
    TL_CUDA_TRY_STATUS(launch_prep_spin2(p, nullptr, nullptr, s));
    TL_CUDA_TRY_STATUS(launch_legendre_adj2(p, 0, p->d7_Q, p->d7_U, alm_E, alm_B, s));
  }
  TL_CUDA_TRY_STATUS(launch_adj_finish(p, alm_T, nullptr, want_pol ? alm_E : nullptr, want_pol ? alm_B : nullptr, s));
  const double w = 4.0 * 3.14159265358979323846 / (double)p->npix;
  dim3 grid((p->lmax + 1 + 127) / 128, p->lmax + 1);
  map2alm_weight_kernel<<<grid, 128, 0, s>>>(p->lmax, w, alm_T);
  if (want_pol) {
    map2alm_weight_kernel<<<grid, 128, 0, s>>>(p->lmax, w, alm_E);
    map2alm_weight_kernel<<<grid, 128, 0, s>>>(p->lmax, w, alm_B);
  }
  TL_CUDA_TRY_STATUS(cudaGetLastError());
  return TL_OK;
}

extern "C" tl_status tl_anafast(int lmax, const double *alm_T, const double *alm_E, const double *alm_B, double *cl,
                                void *stream) {
  if (lmax < 0 || !cl || (!alm_T && !alm_E && !alm_B)) return TL_ERR_ARG;
  const void *ptrs[] = {alm_T, alm_E, alm_B, cl};
  for (const void *q : ptrs)
    if (q && !al16(q)) return TL_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  TL_CUDA_TRY_STATUS(cudaMemsetAsync(cl, 0, sizeof(double) * 6 * (size_t)(lmax + 1), s));
  anafast_kernel<<<(lmax + 1 + 127) / 128, 128, 0, s>>>(lmax, alm_T, alm_E, alm_B, cl);
  TL_CUDA_TRY_STATUS(cudaGetLastError());
  return TL_OK;
}
