/*
 * taylens.h -- C ABI of the GB300 (sm_103a) full-sky Taylor-lensing library.
 *
 * Method: Naess & Louis 2013, "Lensing simulations by Taylor expansion -- not so
 * inefficient after all" (arXiv:1307.0719). The library computes, on one GPU,
 *   - the unlensed T and Q/U maps and all their mixed theta/phi derivative maps
 *     d_theta^j d_phi^k s, j + k <= n, on the HEALPix RING grid (Sec. II.B, Eq. 4),
 *   - the deflection alpha = grad(phi) (Sec. I, Eqs. 1-2; Sec. II.A),
 *   - the lensed maps by the pixel-relative Taylor expansion around the centre of
 *     the pixel containing the displaced point x + alpha (Sec. I, the expansion
 *     after Fig. 1; Sec. II.B, Eq. 4), with the polarisation rotation R of Eq. 2.
 *
 * Conventions shared by every call
 *  - Harmonic coefficients ("alm"): complex128, interleaved (re, im), triangular
 *    layout idx(l, m) = m (2 lmax + 1 - m) / 2 + l for 0 <= m <= l <= lmax
 *    (real fields, m >= 0 only). The imaginary part of m = 0 entries is ignored.
 *    Q +- iU = -sum (E_lm +- i B_lm) +-2Y_lm (HEALPix convention).
 *  - Maps: HEALPix RING order, Npix = 12 nside^2. Element type is double for
 *    TL_FP64 plans and float for TL_MIXED_* plans.
 *  - Every pointer argument named "device" must point to device memory owned by
 *    the caller, 16-byte aligned; the library never frees it. Calls are enqueued
 *    on the given stream (a cudaStream_t passed as void*, NULL = legacy default
 *    stream) and return before the GPU work finishes.
 *  - Errors: every call returns a tl_status. Argument errors are detected on the
 *    host before any GPU work is enqueued. TL_ERR_CUDA reports a failed CUDA
 *    runtime call (launch or allocation); the plan stays valid after argument
 *    errors but should be destroyed after TL_ERR_CUDA.
 *  - A plan may be used by one host thread at a time; different plans are
 *    independent.
 */
#ifndef TAYLENS_H
#define TAYLENS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tl_plan tl_plan; /* opaque; owns its device tables and workspace */

typedef enum {
  TL_OK = 0,
  TL_ERR_ARG = 1,         /* invalid argument (NULL, misaligned, out of range) */
  TL_ERR_NOMEM = 2,       /* device or host allocation failed                  */
  TL_ERR_CUDA = 3,        /* a CUDA runtime call failed                         */
  TL_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up                 */
  TL_ERR_UNSUPPORTED = 5  /* valid request this build does not implement       */
} tl_status;

/* `spins` bitmask */
enum { TL_SPIN_T = 1, TL_SPIN_QU = 2 };

/* `precision`: arithmetic of the Legendre stage, ring FFTs and Taylor sums.
 * TL_FP64          everything in double.
 * TL_MIXED_FP32    float recurrence and contraction with double seeds and
 *                  exponent rescaling; float maps; float pixel lookup with a
 *                  double fallback near cell edges.
 * TL_MIXED_TF32    as TL_MIXED_FP32, but tl_lens / tl_lens_batch contract the
 *                  recurrence against the coefficients on the tensor cores
 *                  (tcgen05, accumulators in tensor memory) in TF32 (10-bit
 *                  mantissas, FP32 accumulation), up to sixteen realisations
 *                  per Legendre launch.
 * TL_MIXED_TF32x3  the same with each operand split into TF32 hi + lo parts and
 *                  three products accumulated (errors close to FP32).
 * TL_MIXED_BF16x3  the same with each operand split into BF16 hi + lo parts
 *                  (8 significant bits each) and the products hi.hi, lo.hi,
 *                  hi.lo and lo.lo accumulated by two K = 16 BF16 MMAs per
 *                  8 values of l.
 * tl_synth_derivs and tl_deflection use the float (SIMT) stage in all mixed forms. */
enum { TL_FP64 = 0, TL_MIXED_FP32 = 1, TL_MIXED_TF32 = 2, TL_MIXED_TF32x3 = 3, TL_MIXED_BF16x3 = 4 };

/* `flags`
 *   TL_ROTATE          apply the polarisation rotation R of Eq. 2 (default on).
 *   TL_NAIVE           the displaced position by naive coordinate addition,
 *                      theta' = theta + alpha_theta, phi' = phi + alpha_phi / sin theta
 *                      (Sec. II.A's alternative to parallel transport; a point carried
 *                      past a pole continues on the other side), instead of the end of
 *                      the geodesic from x along alpha. R keeps the geodesic angle.
 *   TL_EXPAND_AT_PIXEL the Taylor series about the output pixel itself (Sec. I, Eq. 3a:
 *                      the plain expansion about the undisplaced point, the paper's
 *                      motivating comparison) instead of about the centre of the pixel
 *                      containing x' (Sec. II.B).
 * tl_lens_adjoint supports TL_ROTATE only (TL_ERR_UNSUPPORTED otherwise). */
enum { TL_ROTATE = 1, TL_NAIVE = 2, TL_EXPAND_AT_PIXEL = 4 };

/*
 * Create a plan for one (nside, lmax, order) geometry.
 *   nside     power of two, 1 .. 8192
 *   lmax      1 .. 8 nside (band limit of every field, and of phi unless
 *             tl_plan_set_lmax_phi gives it its own)
 *   order     Taylor order n, 0 .. 6 (total degree j + k <= n; 0 = nearest-pixel lookup)
 *   spins     TL_SPIN_T, TL_SPIN_QU or both
 *   precision TL_FP64, TL_MIXED_FP32, TL_MIXED_TF32, TL_MIXED_TF32x3 or
 *             TL_MIXED_BF16x3
 *   flags     any of TL_ROTATE, TL_NAIVE, TL_EXPAND_AT_PIXEL
 *   out       receives the plan; unchanged on error
 * Allocates the plan's device tables and workspace on the current device.
 * Errors: TL_ERR_ARG, TL_ERR_UNSUPPORTED, TL_ERR_NOMEM, TL_ERR_CUDA.
 */
tl_status tl_plan_create(int nside, int lmax, int order, int spins, int precision, int flags,
                         tl_plan **out);

/* Free a plan (synchronises the device first). NULL is accepted. */
tl_status tl_plan_destroy(tl_plan *plan);

/* Device bytes held by the plan (tables + workspace). 0 for NULL. */
size_t tl_plan_workspace_bytes(const tl_plan *plan);

/* Number of derivative maps per field, (order+1)(order+2)/2. */
int tl_plan_maps_per_field(const tl_plan *plan);

/* Realisations that share one Legendre launch in tl_lens_batch: 16 on the
 * tensor-core precisions up to order 5 (8 at order 6), 1 otherwise. Batches of
 * this size use the contraction best. 0 for NULL. */
int tl_plan_batch(const tl_plan *plan);

/* Kernel launches that tl_lens_batch makes for nreal realisations (with the
 * lensing potential when with_phi != 0): the Legendre stage per batch, the ring
 * FFTs (one launch per ring group) and the gather per realisation. -1 for NULL. */
long long tl_plan_batch_launches(const tl_plan *plan, int nreal, int with_phi);

/*
 * Derivative maps of one field (Sec. II.B, Eq. 4: the maps d_theta^j d_phi^k s
 * evaluated at every pixel centre), in natural units.
 *   alm   device; spin 0: nalm complex (T); spin 2: 2*nalm complex, E then B
 *   spin  0 or 2 (the plan must include that field)
 *   maps  device, [K][Npix] with K = maps_per_field (spin 0) or 2*maps_per_field
 *         (spin 2: all Q maps, then all U maps). Map index of (j, k) inside a
 *         field is (j+k)(j+k+1)/2 + j.
 */
tl_status tl_synth_derivs(tl_plan *plan, const double *alm, int spin, void *maps, void *stream);

/*
 * Deflection field alpha = grad(phi) at every pixel centre (Sec. I, Eqs. 1-2):
 * a_theta = d_theta phi, a_phi = d_phi phi / sin(theta), components on the
 * orthonormal (e_theta, e_phi) basis.
 *   alm_phi  device, nalm complex;  a_theta, a_phi  device, [Npix] each.
 */
tl_status tl_deflection(tl_plan *plan, const double *alm_phi, void *a_theta, void *a_phi,
                        void *stream);

/*
 * Lensed maps (Eqs. 1-2 approximated by Eq. 4 around the pixel containing
 * x + alpha, then the rotation R when the plan has TL_ROTATE).
 *   alm_T, alm_E, alm_B   device, nalm complex each; alm_B may be NULL (B = 0);
 *                         alm_E/alm_B ignored and Q_out/U_out untouched for
 *                         T-only plans; alm_T may be NULL only for QU-only plans
 *   alm_phi               device, nalm complex (may be NULL: no lensing)
 *   T_out, Q_out, U_out   device, [Npix] each in RING order
 */
tl_status tl_lens(tl_plan *plan, const double *alm_T, const double *alm_E, const double *alm_B,
                  const double *alm_phi, void *T_out, void *Q_out, void *U_out, void *stream);

/*
 * Lens nreal realisations of this plan's geometry in one call. Arrays of nreal
 * device pointers (host arrays); entries as in tl_lens; alm_B may be NULL (all
 * B = 0); alm_phi may be NULL (none lensed), otherwise every entry must be set.
 * On tensor-core plans (TL_MIXED_TF32, TL_MIXED_TF32x3, TL_MIXED_BF16x3)
 * realisations go through the Legendre stage tl_plan_batch at a time (16, or 8 at
 * order 6), sharing the recurrence (the coefficient sets of all of them fill the
 * 64 (32) columns of one tensor-core product); ring FFTs and the
 * gather then run per realisation. On other plans this equals nreal calls of
 * tl_lens.
 */
tl_status tl_lens_batch(tl_plan *plan, int nreal, const double *const *alm_T, const double *const *alm_E,
                        const double *const *alm_B, const double *const *alm_phi, void *const *T_out,
                        void *const *Q_out, void *const *U_out, void *stream);

/*
 * tl_lens with HOST buffers: copies the alm from host memory to the plan's
 * device staging area, runs tl_lens, copies the maps back and synchronises the
 * stream before returning. Host buffers should be pinned for full speed.
 * Same layouts as tl_lens; outputs are double (TL_FP64) or float (mixed).
 */
tl_status tl_lens_host(tl_plan *plan, const double *alm_T, const double *alm_E,
                       const double *alm_B, const double *alm_phi, void *T_out, void *Q_out,
                       void *U_out, void *stream);

/*
 * tl_lens_batch with HOST buffers, the call a user with maps and coefficients in
 * host memory makes: arrays (host) of nreal host pointers, layouts as in tl_lens.
 * Each chunk of up to tl_plan_batch(plan) realisations (one Legendre launch on
 * tensor-core plans) is copied to device staging owned by the plan (allocated on
 * the first call and grown when a larger chunk is asked for), lensed with
 * tl_lens_batch on `stream`, and its maps copied back; the call synchronises the
 * stream before it returns. Host buffers should be pinned for full speed.
 * Errors as tl_lens_batch, plus TL_ERR_CUDA if a staging allocation fails.
 */
tl_status tl_lens_batch_host(tl_plan *plan, int nreal, const double *const *alm_T, const double *const *alm_E,
                             const double *const *alm_B, const double *const *alm_phi, void *const *T_out,
                             void *const *Q_out, void *const *U_out, void *stream);

/*
 * Reverse mode of tl_lens (the transpose of its linearisation): gradients of a
 * scalar loss with respect to the coefficients, given its gradients with
 * respect to the lensed maps. Naess & Louis 2013, Sec. II (Eq. 4 and the
 * rotation R of Eq. 2), differentiated step by step: the rotation and the Taylor
 * sum of Eq. 4 at each pixel, the displacement geometry of Sec. II.A, the ring
 * synthesis of the derivative maps and the spherical-harmonic (Legendre) stage.
 * The expansion pixel q(p) of every output pixel is held fixed: the lensed map is
 * piecewise smooth in the deflection and q is constant between its jumps.
 *   alm_T, alm_E, alm_B, alm_phi   device, as in tl_lens (alm_phi NULL: alpha = 0)
 *   gT, gQ, gU     device [npix] dL/dT', dL/dQ', dL/dU' in the plan's map type
 *                  (gQ, gU required for TL_SPIN_QU plans, ignored otherwise)
 *   galm_T, galm_E, galm_B, galm_phi
 *                  device [nalm] complex128 outputs, dL/dRe + i dL/dIm per stored
 *                  coefficient (m >= 0; the imaginary part is 0 at m = 0, where the
 *                  coefficients are real). Any of them may be NULL to skip it;
 *                  galm_E and galm_B must be NULL for TL_SPIN_T plans.
 *   galpha         NULL, or device [2][npix] in the plan's map type: receives
 *                  dL/da_theta and dL/da_phi per pixel (the deflection gradient)
 *   stream         cudaStream_t (NULL: legacy default stream)
 * The forward lens is recomputed inside the call. The displacement geometry and
 * its Jacobian are evaluated in double precision for every plan precision.
 * First use allocates the adjoint workspace (the size of the derivative maps
 * plus, without galpha, 2 npix map elements), counted in tl_plan_workspace_bytes.
 * Errors: TL_ERR_ARG for NULL required pointers, misaligned buffers or E/B
 * outputs on a temperature-only plan; TL_ERR_NOMEM, TL_ERR_CUDA as elsewhere.
 */
tl_status tl_lens_adjoint(tl_plan *plan, const double *alm_T, const double *alm_E, const double *alm_B,
                          const double *alm_phi, const void *gT, const void *gQ, const void *gU, double *galm_T,
                          double *galm_E, double *galm_B, double *galm_phi, void *galpha, void *stream);

/*
 * Spherical-harmonic analysis of maps on the plan's geometry (Sec. III: the paper
 * measures the lensed maps through their power spectra, from healpy's map2alm with
 * uniform weights and no iteration, and anafast):
 *   a_lm = (4 pi / Npix) sum_p s(p) conj(sY_lm(p)),
 * s = T (spin 0) and, for Q/U plans, Q +- iU (spin 2) into E and B in the HEALPix
 * convention of tl_synth_derivs (Q + iU = -sum (E + iB) 2Y_lm). This is the
 * transpose of the ring synthesis with those weights (it runs the adjoint kernels
 * of tl_lens_adjoint at order 0), exact for band-limited maps only up to the
 * quadrature error of the HEALPix grid.
 *   T, Q, U        device maps, RING order, the plan's map type (double for TL_FP64,
 *                  float for the mixed forms); Q and U NULL for temperature only
 *   alm_T, E, B    device outputs, complex128 interleaved, healpy order, lmax of the
 *                  plan (E, B NULL when Q, U are)
 * Uses the plan's coefficient planes as workspace (overwrites the last tl_lens's).
 * Errors: TL_ERR_ARG (NULL T or alm_T, unaligned pointers, Q/U on a T-only plan),
 * TL_ERR_CUDA.
 */
tl_status tl_map2alm(tl_plan *plan, const void *T, const void *Q, const void *U, double *alm_T, double *alm_E,
                     double *alm_B, void *stream);

/*
 * Angular power spectra of coefficient sets (Sec. III, Figs. 2, 3, 5, 6):
 *   C_l^XY = (1 / (2l + 1)) sum_{m=-l..l} Re(x_lm conj(y_lm)),   l = 0 .. lmax,
 * real fields (x_l,-m = (-1)^m conj x_lm). cl: device double [6][lmax + 1], rows TT,
 * EE, BB, TE, TB, EB; rows whose fields are NULL are left 0. alm as in tl_map2alm.
 * Errors: TL_ERR_ARG (lmax < 0, NULL cl, no field, unaligned pointers), TL_ERR_CUDA.
 */
tl_status tl_anafast(int lmax, const double *alm_T, const double *alm_E, const double *alm_B, double *cl,
                     void *stream);

/*
 * tl_deflection without any allocation, for callers that cannot allocate device
 * memory while they run (code inside a memory pool or allocator of its own,
 * or a process whose device memory is fixed up front).
 * The paper has no counterpart: this is a deployment variant of tl_deflection
 * and computes the same thing (alpha = grad phi at every pixel centre).
 *   nside      power of two, 1 .. 128
 *   lmax       1 .. min(4 nside, 256)
 *   precision  TL_FP64 (double maps) or TL_MIXED_FP32 (float maps)
 *   alm_phi, a_theta, a_phi   device, 16-byte aligned, as in tl_deflection
 * Larger sizes return TL_ERR_ARG.
 * All tables and working memory sit in one fixed 8 MiB device array inside the
 * library (held by every GPU that loads it, until the process exits); no call
 * allocates device or host memory. The first call on a device, and any call
 * with a different (nside, lmax, precision) than the previous call on that
 * device, first waits for all earlier work on the device (cudaDeviceSynchronize,
 * so that kernels of earlier calls still queued on any stream have finished
 * reading the array) and then lays the tables out in that array with
 * synchronous copies and kernels on the legacy default stream: make that first
 * call before any stream capture. A captured call stays valid only until a call
 * with a different (nside, lmax, precision) is made on that device, which lays
 * the array out again. Every call on a device shares the array and overwrites
 * what the previous call left there, so calls that overlap on the GPU (other
 * streams, other host threads) race; issue them one after another. Not
 * thread-safe.
 */
tl_status tl_deflection_noalloc(int nside, int lmax, int precision, const double *alm_phi,
                                void *a_theta, void *a_phi, void *stream);

/*
 * Batches of realisations of uneven size (different nside / lmax), same order,
 * fields, precision and flags. The batch groups realisations by geometry and
 * owns one plan per group.
 *   tl_batch_create: nreal realisations, nside[i], lmax[i] (host arrays).
 *   tl_batch_lens modes:
 *     TL_BATCH_LOOP        one tl_lens call per realisation (the comparison point);
 *     TL_BATCH_PERSISTENT  tensor-core plans only: waves of up to tl_plan_batch realisations per group, each
 *                          wave's Legendre stage in one persistent launch whose
 *                          blocks take (plan, spin, m, ring block) items, sorted
 *                          by cost, from an atomic counter (no waits between blocks);
 *     TL_BATCH_GRAPH       the persistent sequence captured once as a CUDA graph per
 *                          set of buffer pointers and replayed on `stream`.
 *   The persistent and graph modes need the lensing potential for every realisation
 *   (else TL_ERR_UNSUPPORTED); on non-tensor-core plans they run the loop.
 *   Arrays (host) of nreal device pointers, layouts as in tl_lens.
 *   tl_batch_autotune: times the persistent grid size and the ring-FFT batching
 *   on the given data (synchronises), keeps the fastest, and appends it to the file
 *   named by TAYLENS_TUNE_CACHE when set; tl_batch_create reads that file.
 */
typedef struct tl_batch tl_batch;
enum { TL_BATCH_LOOP = 0, TL_BATCH_PERSISTENT = 1, TL_BATCH_GRAPH = 2 };
tl_status tl_batch_create(int nreal, const int *nside, const int *lmax, int order, int spins, int precision,
                          int flags, tl_batch **out);
tl_status tl_batch_destroy(tl_batch *batch);
tl_status tl_batch_lens(tl_batch *batch, int mode, const double *const *alm_T, const double *const *alm_E,
                        const double *const *alm_B, const double *const *alm_phi, void *const *T_out,
                        void *const *Q_out, void *const *U_out, void *stream);
tl_status tl_batch_autotune(tl_batch *batch, const double *const *alm_T, const double *const *alm_E,
                            const double *const *alm_B, const double *const *alm_phi, void *const *T_out,
                            void *const *Q_out, void *const *U_out, void *stream);
int tl_batch_groups(const tl_batch *batch); /* number of geometry groups */
int tl_batch_waves(const tl_batch *batch);  /* waves of the persistent mode */
int tl_batch_grid(const tl_batch *batch);   /* persistent grid size in use */

/*
 * Device-side error check: synchronises the device and returns TL_ERR_TIMEOUT if
 * a kernel of this plan gave up a bounded wait since the last check (the flag is
 * then cleared), else TL_OK. Kernels that time out record the flag, wait (bounded)
 * for their own tensor-core work, free their tensor memory and return; their
 * outputs are then undefined. TL_ERR_CUDA if the device reports an error.
 */
tl_status tl_plan_device_error(tl_plan *plan);

/*
 * Limit of the bounded waits of the tensor-core kernels (the paper has no
 * counterpart: a control of this implementation's pipeline). Every mbarrier wait
 * of a later launch of this plan polls at most `polls` times (0 restores the
 * default, 2^24) before it gives up as tl_plan_device_error describes. stall = 1
 * is a self-test of that path: the compute warps withhold their arrivals on the
 * tile barriers, so the waits of the next launches run out (nothing faults or
 * hangs: every wait is bounded) and their outputs are undefined; stall = 0
 * restores normal operation. TL_ERR_ARG for polls < 0 or stall not 0 or 1.
 */
tl_status tl_plan_set_wait_limit(tl_plan *plan, int polls, int stall);

/* Band limit of the lensing potential (Sec. II.A: the paper takes the gradient map
 * to min(8 Nside, 10000), above the fields' lmax, since the gradient is sensitive
 * to small scales). Default: the plan's lmax.
 *   lmax_phi  1 .. 8 nside. Any other value than the plan's lmax attaches a deflection plan
 *             at (nside, lmax_phi, order 1, temperature only; the single-precision
 *             SIMT form for every mixed form, FP64 for FP64), which then computes
 *             alpha for every tl_lens, tl_lens_batch, tl_lens_host,
 *             tl_lens_batch_host and tl_deflection call; lmax_phi = lmax removes it.
 * After it, every alm_phi argument holds (lmax_phi+1)(lmax_phi+2)/2 coefficients
 * (healpy order for lmax_phi); the other fields keep the plan's lmax.
 * tl_lens_adjoint returns TL_ERR_UNSUPPORTED while a separate lmax_phi is set.
 * The call waits for the device (work queued on any stream may still use the
 * previous deflection plan) and frees the host-call staging, which the next host
 * call allocates again. Errors: TL_ERR_ARG for a NULL plan or lmax_phi < 1; the
 * errors of tl_plan_create (the plan keeps lmax_phi = lmax then).
 */
tl_status tl_plan_set_lmax_phi(tl_plan *plan, int lmax_phi);

/* Human-readable text for a status code (static storage). */
const char *tl_status_string(tl_status status);

/* Milliseconds of the stages of the most recent tl_lens or tl_lens_adjoint on
 * this plan, measured with CUDA events on the call's stream when the environment
 * variable TAYLENS_TIMING=1 was set at plan creation (otherwise returns 0).
 * tl_lens stage order: prep_T (T and phi coefficients), legendre_T (spin-0 stage,
 * with phi's j <= 1 planes), deflection_fft, prep_QU, legendre_QU, ringfft (all
 * T/Q/U maps), gather, then two totals: all ring FFTs and all gathers of the call
 * (on tensor-core plans the ringfft stage spans every realisation's ring FFTs and
 * gathers, and the deflection_fft and gather stages are empty; the totals
 * separate them; prep_T holds the temperature's coefficient tiles only, and the
 * potential's tiles are prepared inside legendre_T, after the temperature's launch). tl_lens_adjoint: forward (recomputed derivative maps and
 * deflection), gather (transposed), ringfft (transposed), legendre_T (transposed,
 * with phi), legendre_QU (transposed), finish. Synchronises on the last event.
 * Returns the number of stages written (<= n). */
int tl_last_stage_ms(const tl_plan *plan, float *ms, int n);

#ifdef __cplusplus
}
#endif
#endif /* TAYLENS_H */
