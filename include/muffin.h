/*
 * muffin.h -- C ABI of the GB300 (sm_103a) MUFFIN library.
 *
 * MUFFIN (Ammanouil, Ferrari, Mary, Ferrari, Loi 2019) restores a
 * multispectral sky cube X (L bands of n x n pixels) from dirty images
 * Y = H X* + W by minimising (Eqs. probopt, RegAll)
 *
 *   sum_l 1/2 ||y_l - H_l x_l||^2 + 1_{R+}(X)
 *       + sum_l mu_l ||W_s x_l||_1 + sum_n gamma_n ||W_lambda x^n||_1
 *
 * with the primal-dual (Vu-Condat) iteration of Algorithm 2, and tunes the
 * two regularisation weights (mu, gamma) online with ADA-PT (Algorithm 5):
 * SUGAR-FDMC gradients (Eq. SUGAR) of the PSURE-FDMC risk (Eq. PSURE0) from
 * the derivative iterates of Algorithms 3 and 4.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Cubes are float32, band-major, row-major: element (l, y, x) at
 *   l*n*n + y*n + x.  H_l is the circular convolution by psf_l with the PSF
 *   origin at pixel (0, 0) (Eq. model).  W_s is the unscaled union of the
 *   periodised orthonormal Daubechies bases db1..dbK with J levels (Sec.
 *   4.2.1); W_lambda is the orthonormal DCT-II along bands.
 * - mu_l = mu * beta_l and gamma_n = gamma * alpha_n (Eq. 2regpar).
 * - Array arguments may live in host memory or in device memory of the
 *   plan's device; the library detects which (cudaPointerGetAttributes).
 *   Host arrays are copied in and out synchronously inside the call.
 *   Device arrays are read/written on the plan's stream.
 * - The caller owns every array it passes; the plan owns its internal state
 *   (primal/dual iterates, spectra, scratch) and frees it in
 *   muffin_plan_destroy.
 * - Every call returns a status; on failure muffin_last_error() describes
 *   it.  After MUFFIN_ECUDA the plan must be destroyed.  Calls are
 *   synchronous (the plan's stream is synchronised before returning), and a
 *   plan must not be used from two threads at once.
 */
#ifndef MUFFIN_H
#define MUFFIN_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MUFFIN_API __attribute__((visibility("default")))
#else
#define MUFFIN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct muffin_plan_s *muffin_plan;

typedef enum {
  MUFFIN_OK = 0,
  MUFFIN_EINVAL = 1,   /* invalid argument or shape */
  MUFFIN_ENOMEM = 2,   /* device or host allocation failed */
  MUFFIN_ECUDA = 3,    /* CUDA runtime error; destroy the plan */
  MUFFIN_ETIMEOUT = 4, /* a bounded device wait gave up */
  MUFFIN_ENUMERIC = 5, /* NaN/Inf detected in the state */
  MUFFIN_ESTATE = 6    /* call not valid in the plan's current state */
} muffin_status;

/* Plan parameters (Sec. 2.2 step condition, Sec. 4.2.1 settings). */
typedef struct {
  int32_t n;          /* image side, power of two, 2 <= n <= 2048 */
  int32_t nbands;     /* L >= 1 */
  int32_t n_wavelets; /* K in 1..8: W_s = [db1; ...; dbK] (default 8) */
  int32_t levels;     /* J >= 0 with 2^J <= n (default 3); 0 = identity bases */
  double sigma;       /* dual step sigma > 0 (default 10, Sec. 4.2.1) */
  int32_t step_rule;  /* 0: tau from the paper's sum form (default);
                         1: from ||L||^2 = K max mu_l^2 + max gamma_n^2 */
  double tau_safety;  /* tau = safety / (beta/2 + sigma ||L||^2), default 0.99 */
  int32_t positivity; /* 1 (default): projection of Eq. projpos; 0 skips it */
  int32_t sure;       /* 1: also allocate the ADA-PT chains (needed by
                         muffin_sure_tune); 0: plain MUFFIN only */
  int32_t batch;      /* B >= 1 independent cubes of the same shape advanced
                         by the same launches (default 1); every cube array
                         argument below then holds B cubes one after the
                         other: [B][L][n][n] */
  int32_t dictionary; /* spatial dictionary W_s (Sec. 2.1): 0 = union of the
                         first n_wavelets Daubechies bases (default), K =
                         n_wavelets coefficient planes per band, ||W_s||^2 =
                         K; 1 = isotropic undecimated wavelet transform
                         (starlet, B3 spline, periodic) with J = levels <= 4
                         scales, K = J + 1 planes, ||W_s||^2 = 1 */
  int32_t precision;  /* arithmetic of the spectral DCT W_lambda (Sec. 4.2.1):
                         0 (default) = dense L x L products as 3xTF32 split
                         products on the tensor cores, FP32 accumulation;
                         1 = FP32 on the CUDA cores by a fast DCT-II
                         (Makhoul's reordering into one complex DFT per
                         pixel, O(L log L)); needs nbands a power of two in
                         [2, 1024] */
  double tau;         /* primal step override: > 0 makes every solve and
                         every ADA-PT window use this tau instead of the
                         step rule (the caller then answers for the step
                         condition of Sec. 2.2); 0 (default) = from
                         step_rule and tau_safety */
} muffin_params;

/* Fill *p with the defaults above for an n x n x nbands cube. */
MUFFIN_API void muffin_params_default(muffin_params *p, int32_t n, int32_t nbands);

/*
 * Create a plan: validates p, allocates the device state, computes the PSF
 * spectra h_hat_l = F psf_l (FP64), beta = max_l ||H_l||^2 =
 * max_{l,k} |h_hat_l(k)|^2 per cube (the Lipschitz constant of the
 * least-squares gradient, Sec. 2.2), the Daubechies filters and the DCT-II
 * tables.
 *   psf   [B][L][n][n] float32, host or device; read during the call only.
 *   alpha [B][n*n] pixel weights alpha_n, or NULL for all ones (Eq. 2regpar).
 *   beta  [B][L]   band weights beta_l, or NULL for all ones.
 *   stream  a cudaStream_t (NULL = legacy default stream) used for all work.
 * Errors: EINVAL (shape, NULL out, PSF all zero), ENOMEM, ECUDA.
 */
MUFFIN_API muffin_status muffin_plan_create(const muffin_params *p, const float *psf,
                                 const float *alpha, const float *beta,
                                 void *stream, muffin_plan *out);

MUFFIN_API void muffin_plan_destroy(muffin_plan plan);

/* Device bytes held by the plan (state + scratch). */
MUFFIN_API size_t muffin_plan_device_bytes(muffin_plan plan);

/* beta[b] = max_l ||H_l||^2 of cube b (FP64), b < B. */
MUFFIN_API muffin_status muffin_plan_lipschitz(muffin_plan plan, double *beta);

/* Device bytes muffin_plan_create would allocate for p (the footprint used
 * for admission by the request server).  Errors: EINVAL for invalid p. */
MUFFIN_API muffin_status muffin_plan_estimate_bytes(const muffin_params *p,
                                                    size_t *bytes);

/* Replace the PSFs of cubes [b0, b1): psf [b1-b0][L][n][n] (host or device);
 * recomputes their spectra and beta (the state is kept). */
MUFFIN_API muffin_status muffin_plan_load_psf(muffin_plan plan, int32_t b0,
                                              int32_t b1, const float *psf);

/*
 * Visibility-domain data term (Sec. 1: the method applies unchanged when the
 * direct operator maps the sky to its visibilities).  Reading: the
 * visibilities of band l sample the unitary 2D DFT U = F / n of x_l on the
 * n x n grid (nearest cell), and the data term is
 * 1/2 sum_p |d_p - (U x_l)_{k(p)}|^2; gridded into per-cell sums D_l[k] and
 * natural weights m_l[k] (sample counts), its gradient for real x is
 *   F^-1 (m~_l . F x_l) - Re U^H D_l,   m~_l[k] = (m_l[k] + m_l[-k]) / 2.
 * The call replaces every cube's PSF spectra by h_hat_l = sqrt(m~_l) and
 * b = H^T y by Re U^H D_l (FP64), and recomputes beta = max m~; a following
 * muffin_solve / muffin_solve_batch with dirty = NULL then runs Algorithm 2
 * on this data term from the given X0 (a dirty cube passed to a later call
 * returns the plan to the image-domain model with the current spectra; a
 * PSF load replaces them).
 *   vis     [B][L][n][n][2] float32 (re, im) per-cell sums D, host or device,
 *           cell (ky, kx) at index ky * n + kx (FFT order, DC at 0);
 *   weights [B][L][n][n] float32 m >= 0, host or device.
 * Both are read during the call only.  ADA-PT and the monitor's objective
 * need a dirty cube (they return EINVAL / ESTATE for this data term).
 * Errors: EINVAL (NULL, a negative, NaN or Inf weight, all weights of a
 * cube zero), ENUMERIC (NaN/Inf visibility), ECUDA.
 */
MUFFIN_API muffin_status muffin_plan_load_visibilities(muffin_plan plan, const float *vis,
                                                       const float *weights);

/* on = 1 (default): repeated launch sequences (two plain iterations, one
 * ADA-PT window) are captured once into CUDA graphs and replayed; 0 launches
 * every kernel directly.  Results are identical either way. */
MUFFIN_API muffin_status muffin_plan_graphs(muffin_plan plan, int32_t on);

/* ---- weights (Eq. 2regpar)
 *
 * mu_l = mu beta_l and gamma_n = gamma alpha_n.  Replaces the plan's weights:
 *   alpha [B][n*n], beta [B][L] (host or device arrays, >= 0, finite); NULL
 *   keeps the current values.  The step condition (tau) follows the new
 *   weights from the next call on.  Errors: EINVAL (NULL plan, bad value). */
MUFFIN_API muffin_status muffin_plan_set_weights(muffin_plan plan, const float *alpha,
                                                 const float *beta);

/* Weights from an initial cube x0 [B][L][n][n] (host or device), as defined
 * right after Eq. 2regpar:
 *   alpha_n = 1 / (||W_lambda (x^n)_0||_2 + eps_alpha)   (pixel spectra)
 *   beta_l  = 1 / (||W_s (x_l)_0||_2 + eps_beta)          (band images)
 * computed with Parseval's identity (the DCT and each of the K bases are
 * orthonormal, so ||W_lambda x^n|| = ||x^n|| and ||W_s x_l|| = sqrt(K) ||x_l||)
 * in FP64, rounded to FP32, and installed in the plan as by
 * muffin_plan_set_weights.  A coarse x0 is, e.g., a few plain iterations.
 * alpha_out [B][n*n] and beta_out [B][L] (host or device) receive the
 * weights when not NULL.  Errors: EINVAL (NULL plan or x0, eps < 0 or not
 * finite), ECUDA. */
MUFFIN_API muffin_status muffin_plan_weights_from_x0(muffin_plan plan, const float *x0,
                                                     double eps_alpha, double eps_beta,
                                                     float *alpha_out, float *beta_out);

/* ---- per-shape tuning (launch variants of the hot kernels)
 *
 * For 64-band plans the tuner also times the two spectral kernels (tcgen05
 * and mma.sync), whose results agree to FP32 accuracy.  Two further launch
 * choices change speed but not results (every variant computes the same
 * sums in the same order, so outputs are bit-identical):
 *   syn_packed       bit 0: coarse wavelet synthesis levels, bit 1: level 1;
 *                    0 = scalar row pass (one pixel row per thread),
 *                    1 = packed row pass (two rows per fma.rn.f32x2);
 *   dct_ctas_per_sm  CTAs per SM of the persistent spectral kernel
 *                    (0 = as many as fit).
 * Which is fastest depends on the cube shape and the GPU. */
typedef struct {
  int32_t syn_packed;      /* chosen synthesis variant bits */
  int32_t dct_ctas_per_sm; /* chosen grid of the mma.sync spectral kernel (0 = all resident) */
  int32_t spectral_tcgen05;/* 1: spectral step on tcgen05 (64-band plans, see
                              muffin_plan_set_spectral_kernel) */
  int32_t from_cache;      /* 1: taken from the in-process or file cache */
  int32_t candidates;      /* configurations timed (0 when cached) */
  double ms_default;       /* one iteration of every chain group, default */
  double ms_best;          /* the same with the chosen variants */
  int32_t grad_chunk;      /* chosen gradient chunking (muffin_schedule) */
  int32_t fft_radix;       /* chosen FFT plan */
  int32_t group_order;     /* chosen kernel order of the ADA-PT groups */
  int32_t ana_ring;        /* chosen analysis U staging */
  int32_t ana_pipe;        /* chosen level-1 analysis kernel */
} muffin_tune_info;

/* Times each candidate configuration on this plan's own buffers (a few
 * iterations of every chain group it advances: two groups of three chains
 * with sure = 1, one plain group otherwise), keeps the fastest and caches it
 * per shape (n, bands, batch, chains, levels, bases, spectral precision, SM
 * count, device name): in process, and in the text file `cache_path` when it
 * is not NULL (read first, one line "muffin-tune-6 <key> <syn_packed>
 * <dct_ctas> <tcgen05> <grad_chunk> <fft_radix> <group_order> <ana_ring>
 * <ana_pipe>"
 * appended per new shape; lines that do not parse are ignored).  The timing iterations overwrite the plan's iterate state: a
 * following solve or sure_tune must start cold (warm = 0; a warm call
 * returns MUFFIN_ESTATE), and captured graphs are rebuilt.  info may be NULL.
 * Errors: EINVAL (plan NULL), ECUDA. */
MUFFIN_API muffin_status muffin_plan_autotune(muffin_plan plan, const char *cache_path,
                                              muffin_tune_info *info);

/* Spectral step kernel for plans with 64 bands: 1 (default for L = 64) runs
 * it on the tcgen05 tensor cores (tensor-memory accumulators, operands in
 * shared memory), 0 on the warp-level mma.sync kernel used for other band
 * counts.  Both compute the same 3xTF32 products; their FP32 rounding order
 * differs, so results agree to FP32 accuracy, not bit for bit.  Drops
 * captured graphs and the iterate state.  Errors: EINVAL (NULL plan, or 1
 * with L != 64). */
MUFFIN_API muffin_status muffin_plan_set_spectral_kernel(muffin_plan plan, int32_t tcgen05);

/* Failure-path test hook (the paper has no counterpart).  on = 1 makes the
 * tcgen05 spectral kernel skip its tensor-core products, so its bounded
 * waits on their completion run out: the kernel raises the plan's error
 * flag, frees its tensor memory and returns, and the next call that
 * synchronises (solve, sure_tune, ...) returns MUFFIN_ETIMEOUT; the results
 * of that call are unspecified and the plan stays usable.  Only plans whose
 * spectral step runs on tcgen05 (64 bands) wait on the device at all.
 * on = 0 restores normal operation.  Drops captured graphs and the iterate
 * state.  Errors: EINVAL (NULL plan). */
MUFFIN_API muffin_status muffin_plan_inject_timeout(muffin_plan plan, int32_t on);

/* Sets the variants directly (syn_packed in 0..3, dct_ctas_per_sm >= 0);
 * drops captured graphs.  Errors: EINVAL. */
MUFFIN_API muffin_status muffin_plan_set_tuning(muffin_plan plan, int32_t syn_packed,
                                                int32_t dct_ctas_per_sm);

/* Every launch choice of the per-iteration schedule (what the tuner picks).
 * None changes results except spectral_tcgen05 and fft_radix (FP32 rounding
 * order; both variants stay within the same tolerance of the oracle). */
typedef struct {
  int32_t syn_packed;       /* synthesis row-pass variant bits, 0..3 */
  int32_t dct_ctas_per_sm;  /* mma.sync spectral grid, 0 = all resident */
  int32_t spectral_tcgen05; /* 64-band plans: 1 tcgen05, 0 mma.sync */
  int32_t grad_chunk;       /* images per pass of the gradient's three FFT
                               passes: 0 = each pass over all images of a
                               chain group; k > 0 = the three passes run k
                               images at a time, so the spectra stay in L2 */
  int32_t fft_radix;        /* largest radix of the gradient's FFT plan: 16
                               (default) or 8 (n >= 64; 1024 = 8.8.8.2 instead
                               of 16.16.4); results agree to FP32 rounding */
  int32_t group_order;      /* ADA-PT plans: 0 = one chain group's kernels
                               after the other's, 1 = both groups phase by
                               phase, 2 = the two groups concurrently on two
                               streams, each with its own scratch (identical
                               results) */
  int32_t ana_ring;         /* analysis of the levels specialised for 512,
                               1024 and 2048 px: 0 = the dual update's U
                               values loaded by each thread, 1 = the U detail
                               tiles staged two steps ahead in a shared-memory
                               ring by cp.async (3 CTAs per SM instead of 4;
                               identical results) */
  int32_t ana_pipe;         /* level-1 analysis of an iteration (levels > 1):
                               0 (default) = basis-major steps with two
                               barriers each; 1 = chain-major steps with the
                               row pass of one step and the column pass +
                               dual update of the previous one in the same
                               phase (two lo/hi buffers, one barrier per
                               step); identical results */
} muffin_schedule;

/* Reads / sets the schedule (set drops captured graphs and the iterate
 * state).  Errors: EINVAL (NULL, a value out of range). */
MUFFIN_API muffin_status muffin_plan_get_schedule(muffin_plan plan, muffin_schedule *s);
MUFFIN_API muffin_status muffin_plan_set_schedule(muffin_plan plan, const muffin_schedule *s);

typedef struct {
  int32_t iters_done; /* iterations run by this call */
  double tau;         /* primal step used (last window for ADA-PT) */
  double sigma;       /* dual step */
  double lipschitz;   /* beta */
  double mu, gamma;   /* regularisation weights at the end of the call */
  int32_t records;    /* ADA-PT trace records written by this call */
  int32_t checks;     /* convergence-monitor checks made by this call */
  int32_t stopped_early; /* 1: the monitor's rel_tol ended the call early */
  double rel_change;  /* last check, cube 0: ||X^k - X^{k-1}|| / ||X^{k-1}||
                         (NaN without checks) */
  double objective;   /* last check, cube 0: the objective (NaN if not asked) */
} muffin_info;

/* ---- convergence monitor (Sec. 2.1: the iteration has no closed form and
 * is run until it settles; Sec. 3.3 monitors the iterates the same way)
 *
 * Every call of muffin_solve / muffin_sure_tune ends with an FP64 scan of the
 * restored cube for NaN/Inf: if one is found the call returns
 * MUFFIN_ENUMERIC, the caller's x holds the non-finite cube, and the plan
 * forgets its iterate state (the next call must start cold, which works
 * normally).  With monitoring on, the plan also checks the iterates of the
 * primal chain on y after every `every` iterations (at the first window end
 * at or after it for muffin_sure_tune), in FP64:
 *   rel_change = ||X^k - X^{k-1}||_2 / ||X^{k-1}||_2 (inf when X^{k-1} = 0
 *                and X^k != 0; 0 when both are 0),
 *   objective  = sum_l 1/2 ||y_l - H_l x_l||^2 + sum_l mu_l ||W_s x_l||_1
 *                + sum_n gamma_n ||W_lambda x^n||_1   (Eqs. probopt, RegAll;
 *                X >= 0 always holds for the iterates), with the call's
 *                (mu, gamma) (for ADA-PT the values after that window's
 *                update), the residual from an FP64 convolution,
 *   and the NaN/Inf scan (MUFFIN_ENUMERIC as above, at once).
 * A check synchronises the plan's stream.  With rel_tol > 0 the call stops
 * after the first check at which every cube has rel_change <= rel_tol
 * (info->stopped_early = 1, info->iters_done = the iterations run). */
typedef struct {
  int32_t every;      /* K >= 1: check every K iterations; 0: end scan only */
  int32_t objective;  /* 1: evaluate the objective at each check (keeps a
                         device copy of the dirty cube, loaded by the next
                         call that passes one) */
  double rel_tol;     /* > 0: early exit as above; 0: fixed iteration count */
} muffin_monitor_params;

typedef struct {
  int32_t k;          /* iterations completed by the call at the check */
  int32_t cube;       /* cube index b < B */
  double rel_change;  /* as above */
  double objective;   /* as above, NaN when not evaluated */
  int64_t nonfinite;  /* NaN/Inf entries of X^k */
} muffin_monitor_record;

/* mp = NULL switches monitoring off (the end-of-call scan stays).
 * Errors: EINVAL (every < 0, rel_tol < 0 or not finite), ENOMEM, ECUDA. */
MUFFIN_API muffin_status muffin_plan_set_monitor(muffin_plan plan,
                                                 const muffin_monitor_params *mp);
/* The last call's check records (per check, per cube, in order): copies up
 * to capacity, *count = the number recorded.  Errors: EINVAL. */
MUFFIN_API muffin_status muffin_plan_monitor_read(muffin_plan plan,
                                                  muffin_monitor_record *out,
                                                  int32_t capacity, int32_t *count);
/* Objective (Eqs. probopt, RegAll) of a cube x [B][L][n][n] for the dirty
 * cubes [B][L][n][n] (both host or device) and per-cube weights mu[B],
 * gamma[B] (host), with the plan's PSFs and weights alpha_n, beta_l:
 * f[b] (host, B values); +inf for a cube with a negative entry when the plan
 * projects on the positive orthant.  FP64 sums, FP32 transforms.
 * Errors: EINVAL (NULL argument, negative weights), ENOMEM, ECUDA. */
MUFFIN_API muffin_status muffin_objective(muffin_plan plan, const float *dirty,
                                          const float *x, const double *mu,
                                          const double *gamma, double *f);

#define MUFFIN_WARM 1 /* continue from the plan's current state (x ignored
                         on input; dirty may be NULL to keep the last one) */

/*
 * Plain MUFFIN: run `iters` iterations of Algorithm 2 with fixed (mu, gamma)
 * for every cube of the plan.
 *   dirty [B][L][n][n] dirty cubes y (NULL with MUFFIN_WARM: keep the last).
 *   x     [B][L][n][n] in: X0 (ignored with MUFFIN_WARM), out: X after iters.
 *   Without MUFFIN_WARM the duals start at U = V = T = 0.
 *   tau is derived from (mu, gamma) by the plan's step rule.
 *   info  optional (NULL allowed).
 * Errors: EINVAL (iters < 0, NULL x, NULL dirty without warm state, negative
 * mu/gamma), ECUDA.
 */
MUFFIN_API muffin_status muffin_solve(muffin_plan plan, const float *dirty, float *x,
                           int32_t iters, double mu, double gamma,
                           int32_t flags, muffin_info *info);

/* muffin_solve with per-cube weights: mu[B], gamma[B] (host arrays). */
MUFFIN_API muffin_status muffin_solve_batch(muffin_plan plan, const float *dirty,
                                            float *x, int32_t iters,
                                            const double *mu, const double *gamma,
                                            int32_t flags, muffin_info *info);

/* ADA-PT settings (Algorithm 5, Eq. adaptgrad). */
typedef struct {
  int32_t iters;             /* ADA-PT iterations (all 6 chains advance) */
  int32_t window;            /* Delta: theta is updated after every Delta
                                completed iterations (default 10) */
  double eta_mu, eta_gamma;  /* gradient steps for mu and gamma */
  double theta_min;          /* lower clamp of mu and gamma (default 1e-8) */
  int32_t reset_each_window; /* 1 (default): derivative iterates restart at
                                0 at every window; 0 carries them over */
  double eps;                /* FDMC step epsilon > 0 (Eq. PSURE0) */
} muffin_sure_params;

MUFFIN_API void muffin_sure_params_default(muffin_sure_params *s);

/* One record per theta update. */
typedef struct {
  int32_t k;                   /* completed iterations at the update */
  double mu, gamma;            /* theta used during the window */
  double sugar_mu, sugar_gamma;/* Eq. SUGAR summed over bands */
  double psure;                /* Eq. PSURE (per-band noise variances) */
  double tau;                  /* tau used during the window */
} muffin_sure_record;

/*
 * ADA-PT'ed MUFFIN (Algorithm 5): advances the primal chain on y, the
 * primal chain on y_bar = y + eps*delta and the four derivative chains
 * dX/dmu, dX/dgamma, dXbar/dmu, dXbar/dgamma (Algorithms 3, 4) in lockstep;
 * after every `window` iterations computes SUGAR, updates
 * theta <- max(theta - eta * SUGAR, theta_min), recomputes tau and restarts
 * the derivative iterates.
 *   dirty     [B][L][n][n] y.   delta [B][L][n][n] N(0,1) probe.
 *   noise_var [B][L] host array, sigma_l^2 of each band.
 *   x         [B][L][n][n] in: X0 for both primal chains (ignored with
 *             MUFFIN_WARM), out: X of the chain on y.
 *   theta     host double[B][2] in: (mu, gamma) per cube, out: tuned values.
 *   trace     host array [B][iters/window + 1] of records (cube-major), or
 *             NULL; info->records says how many per cube were written.
 * The plan must have been created with p.sure = 1.
 * Errors: EINVAL, ESTATE (plan without SURE chains), ECUDA.
 */
MUFFIN_API muffin_status muffin_sure_tune(muffin_plan plan, const float *dirty,
                               const float *delta, const double *noise_var,
                               const muffin_sure_params *sp, float *x,
                               double *theta, muffin_sure_record *trace,
                               int32_t flags, muffin_info *info);

/* Global SUGAR descent with n_c chosen by the rule of Sec. 3.3 (after Eq.
 * globalgrad): at every outer step, MUFFIN and the derivative chains run
 * from the initial cube with theta fixed, and k -> ||grad R_{0:k}(theta)||
 * (the SUGAR pair, derivatives carried from k = 0) is evaluated every
 * `check` iterations; n_c is the first k >= 2 check with
 *   | ||grad R_{0:k}|| - ||grad R_{0:k-check}|| | <= tol ||grad R_{0:k}||
 * for every cube, or sp->iters (the cap) if that comes first; then
 * theta <- max(theta - eta grad R_{0:n_c}, theta_min).  The cap sp->iters must
 * be a multiple of check.  With tol = 0 the rule never fires and the result
 * is muffin_sure_global's with n_c = sp->iters, up to the rounding of tau
 * (recomputed on the device at every check).  Arguments as
 * muffin_sure_global; trace record i of cube b (at [b][outer]) has k = the
 * n_c used.  Errors: EINVAL (check < 1, tol < 0, cap not a multiple of
 * check, ...), ESTATE, ENOMEM, ECUDA. */
MUFFIN_API muffin_status muffin_sure_global_auto(muffin_plan plan, const float *dirty,
                                                 const float *delta, const double *noise_var,
                                                 const muffin_sure_params *sp, int32_t outer,
                                                 int32_t check, double tol, float *x,
                                                 double *theta, muffin_sure_record *trace,
                                                 muffin_info *info);

/* Global SUGAR descent (Eq. globalgrad): `outer` steps of
 *   theta <- max(theta - eta * SUGAR_{0:n_c}(theta), theta_min)
 * where every step restarts both primal chains from the same initial cube
 * and runs n_c = sp->iters iterations of MUFFIN and of the derivative
 * chains with theta fixed (sp->window is ignored: one window of n_c).
 * Arguments as muffin_sure_tune, plus
 *   outer  number of descent steps (0 leaves x and theta unchanged);
 *   x      in: X0, out: X after the last step's n_c iterations;
 *   trace  host array [B][outer] (cube-major) of one record per step, or NULL.
 * Errors: EINVAL, ESTATE (plan without ADA-PT chains), ENOMEM, ECUDA. */
MUFFIN_API muffin_status muffin_sure_global(muffin_plan plan, const float *dirty,
                                            const float *delta, const double *noise_var,
                                            const muffin_sure_params *sp, int32_t outer,
                                            float *x, double *theta, muffin_sure_record *trace,
                                            muffin_info *info);

/* ---- band-sharded iteration (Sec. 2.3) -----------------------------------
 * The paper distributes an iteration of Algorithm 2 over nodes: the
 * per-band work (eqs. grad2 .. stpu) on slaves that own bands, the per-pixel
 * spectral work (eqs. vt, v, upt) on a master.  These two calls are the
 * halves of one iteration for a band-sharded solve over several GPUs, one
 * process per GPU: between them the caller transposes z = 2 x~ - x from
 * band-sharded to pixel-sharded and t back (one all-to-all each way; the
 * Python driver paper_1905_08468_gb300.sharded does this with
 * torch.distributed).  With every band on one rank the pair computes exactly
 * what muffin_solve's fused iteration does.
 *
 * muffin_shard_spatial: on a plan of this rank's bands (plain, one cube,
 * Daubechies dictionary) whose state was started by muffin_solve(..., iters
 * = 0) (dirty cube, X0, U = V = T = 0):
 *   t     [L][n][n] (host or device): this rank's bands of T from the last
 *         spectral step (zeros before the first);
 *   z     [L][n][n] (host or device) receives z = 2 x~ - x; the plan's X
 *         becomes x~;
 *   mu, gamma, tau: the iteration's weights and primal step (the caller
 *         computes tau from the whole cube's step condition).
 * muffin_shard_spectral: on a plan created for every band of the cube
 * (nbands = the full L; its pixel weights alpha are used, its PSF is not):
 *   for the pixels [p0, p0 + npix) of the image, v <- sat(v + sigma gamma
 *   alpha_n C z^n) and t^n = gamma alpha_n C^T v^n; z, v (in/out), t are
 *   [L][npix] device arrays, 16-byte aligned, npix a multiple of 4.
 * Errors: EINVAL, ESTATE (spatial step before the state was started), ECUDA. */
MUFFIN_API muffin_status muffin_shard_spatial(muffin_plan plan, const float *t, float *z,
                                              double mu, double gamma, double tau);
MUFFIN_API muffin_status muffin_shard_spectral(muffin_plan plan, const float *z, float *v,
                                               float *t, int64_t p0, int64_t npix,
                                               double gamma);

/* ---- noise level ---------------------------------------------------------
 * Sec. 3.1 takes the noise variances as known, or estimated in the image
 * domain by robust statistics such as the median absolute deviation.  Reading
 * (Donoho and Johnstone's wavelet MAD): for every band, the finest diagonal
 * (high-high) band of the orthonormal Haar transform of the dirty image,
 *   d = (y[2i][2j] - y[2i][2j+1] - y[2i+1][2j] + y[2i+1][2j+1]) / 2,
 * sigma_l = median(|d - median(d)|) / 0.6744897501960817 (Phi^-1(3/4)); the
 * median of an even count is the mean of the two middle values (exact order
 * statistics on the FP32 coefficients).  noise_var [B][L] (host) receives
 * sigma_l^2, the form muffin_sure_tune takes.  The estimate assumes the
 * finest scale is dominated by noise; a sky whose convolved image has
 * strong structure at the pixel scale biases it upwards.
 *   dirty [B][L][n][n] (host or device).
 * Errors: EINVAL (NULL argument), ENUMERIC (non-finite input), ECUDA. */
MUFFIN_API muffin_status muffin_noise_mad(muffin_plan plan, const float *dirty,
                                          double *noise_var);

/* ---- checkpoint / resume ------------------------------------------------
 * The state blob holds the iterates (X, U, V, T of every chain), the
 * dirty-cube terms and theta; importing it into a plan created with the
 * same parameters and PSF continues bit-identically (MUFFIN_WARM calls).
 * Blob layout (native byte order), so that the iterates can be inspected:
 *   56-byte header: char magic[8]; int32 n, L, K, J, sure, B; int64 k_done;
 *                   int32 have_b, have_state, have_sure_state, dictionary;
 *   per cube: double {psure constant, mu, gamma};
 *   per chain group g (g = 0 on y; with sure = 1 also g = 1 on
 *   y + eps delta), each of C chains (C = 3 with sure = 1: primal, dX/dmu,
 *   dX/dgamma (Algorithms 3/4); else C = 1), float32 arrays in the order
 *     X [C][B*L][n][n], U [C][B*L][K][n][n], V [C][B*L][n][n], T [C][B*L][n][n];
 *   H^T y [B*L][n][n] float32; with sure = 1 also H^T y_bar and H^T delta;
 *   the per-cube device scalars (4 doubles each: mu, gamma, tau, sigma);
 *   per band 2 sigma_l^2 / eps (double). */
MUFFIN_API muffin_status muffin_state_size(muffin_plan plan, size_t *bytes);
MUFFIN_API muffin_status muffin_state_export(muffin_plan plan, void *host_buf,
                                  size_t bytes);
MUFFIN_API muffin_status muffin_state_import(muffin_plan plan, const void *host_buf,
                                  size_t bytes);

/* ---- single operators, for checking the kernels one by one -------------
 * All cubes [L][n][n] unless stated; coefficients [L][K][n][n] in the Mallat
 * layout of each basis.  They use the same kernels as the iteration. */

/* g = H_l^T (H_l x_l - y_l) per band when dirty != NULL, else H_l^T H_l x_l
 * (Alg. 2 eq. grad2). */
MUFFIN_API muffin_status muffin_op_gradient(muffin_plan plan, const float *x,
                                 const float *dirty, float *g);
/* u = W_s x (analysis over the K bases). */
MUFFIN_API muffin_status muffin_op_analysis(muffin_plan plan, const float *x, float *u);
/* x = W_s^T u (synthesis summed over the K bases). */
MUFFIN_API muffin_status muffin_op_synthesis(muffin_plan plan, const float *u, float *x);
/* v^n = C x^n for every pixel (inverse = 0) or x^n = C^T v^n (inverse = 1),
 * C the orthonormal DCT-II (3xTF32 tensor-core products). */
MUFFIN_API muffin_status muffin_op_dct(muffin_plan plan, const float *x, float *v,
                            int32_t inverse);

/* ---- request server (continuous batching) --------------------------------
 * Deconvolution requests of any shape (n, L) with fixed (mu, gamma) are
 * queued, admitted in arrival order into free slots of batched plans ("pools",
 * one per shape) while the active work stays under max_active_voxels and the
 * pools' device footprint fits the HBM budget, and advanced a chunk of
 * iterations at a time in shared launches.  Pools run independently on their
 * own streams: a pool takes new requests and retires finished ones at its own
 * chunk boundaries, and the pool holding the oldest request runs on the
 * highest-priority stream (the next oldest on the second), so the oldest work
 * gets the GPU first while younger pools fill the rest.  A request's result
 * does not depend on the other requests in its pool.  The caller drives the
 * loop (submit as requests arrive, step, poll).  Not thread-safe: one thread
 * per server. */
typedef struct muffin_server_s *muffin_server;

typedef struct {
  size_t hbm_budget_bytes; /* device bytes the pools may hold; 0 = 80 % of the
                              free device memory at creation */
  int32_t max_batch;       /* slots per pool (default 8) */
  int32_t n_wavelets;      /* K (default 8) */
  int32_t levels;          /* J (default 3) */
  double sigma;            /* dual step (default 10) */
  int32_t step_rule;       /* as muffin_params (default 0) */
  double tau_safety;       /* default 0.99 */
  int32_t chunk;           /* iterations per pool chunk (default 10) */
  size_t max_active_voxels;/* admission stops (in arrival order) once the
                              requests in slots hold this many voxels; one
                              request is always admitted (default 3 * 2^24) */
} muffin_server_params;

MUFFIN_API void muffin_server_params_default(muffin_server_params *p);
/* stream: cudaStream_t the server's work is ordered after (NULL = legacy). */
MUFFIN_API muffin_status muffin_server_create(const muffin_server_params *p,
                                              void *stream, muffin_server *out);
MUFFIN_API void muffin_server_destroy(muffin_server s);
/* Queue a request: psf and dirty [L][n][n] (host or device, copied now;
 * when nothing is queued ahead and an idle pool of its shape has a free slot,
 * the request is admitted at once, straight from these arrays), Algorithm 2
 * with fixed (mu, gamma) from X0 = 0 for `iters` iterations.  A request
 * whose inputs turn out non-finite at admission is rejected: its poll
 * returns MUFFIN_ENUMERIC (or EINVAL for a PSF whose spectrum is not finite)
 * and releases the ticket.  Errors: EINVAL (shape), ENOMEM (one pool of this
 * shape exceeds the budget), ECUDA. */
MUFFIN_API muffin_status muffin_serve_submit(muffin_server s, int32_t n,
                                             int32_t nbands, const float *psf,
                                             const float *dirty, double mu,
                                             double gamma, int32_t iters,
                                             uint64_t *ticket);
/* One scheduling step, without waiting for the slowest pool: collect the
 * pools whose chunk has finished and retire their finished requests, admit
 * queued requests into idle pools, launch the next chunk (up to `chunk`
 * iterations) of every idle pool with active requests.  When none of these
 * happened while chunks are in flight, waits for the first of them to finish
 * and does it again, so every step makes progress.  *active / *queued
 * (nullable) report the requests in slots and still waiting.  Errors: ECUDA,
 * ENOMEM, ETIMEOUT (no chunk finished within 60 s). */
MUFFIN_API muffin_status muffin_serve_step(muffin_server s, int32_t *active,
                                           int32_t *queued);
/* *done = 1 once the request has finished; then, if x_out != NULL, its cube
 * [L][n][n] is copied to x_out (host or device) and the ticket is released.
 * A rejected request (see muffin_serve_submit) returns its error with
 * *done = 1 and releases the ticket. */
MUFFIN_API muffin_status muffin_serve_poll(muffin_server s, uint64_t ticket,
                                           int32_t *done, float *x_out);
/* Device bytes held by the pools and their number (nullable outputs). */
MUFFIN_API muffin_status muffin_server_stats(muffin_server s, size_t *device_bytes,
                                             int32_t *pools);

/* ---- allocation-free operator ------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory: a host program that gives the
 * library a fixed device-memory budget and forbids allocations after
 * start-up, a latency-critical pipeline that cannot afford the implicit
 * device-wide synchronisation cudaMalloc/cudaFree may cause, or code running
 * where the CUDA allocator must not be re-entered (for example inside a
 * memory-pool callback).
 *
 * u = W_s x, exactly what muffin_op_analysis computes, with no plan: x
 * [nbands][n][n] and u [nbands][n_wavelets][n][n] are non-overlapping arrays
 * owned by the caller, in device memory of the current device (or managed
 * memory); the work is enqueued on `stream` (a cudaStream_t, NULL = legacy
 * default stream) and the call returns without synchronising.  Levels 2..J
 * use a fixed file-scope device scratch of 4 Mi floats (16 MiB), which every
 * GPU that loads the library keeps until the process exits; a cube needing
 * more (nbands * n_wavelets * sum_{1<=j<levels} (n>>j)^2 floats) is rejected
 * with MUFFIN_EINVAL before any work.  The call never allocates (no
 * cudaMalloc/cudaFree, no library allocation).  The first call on a device
 * does a one-time set-up with that device current (it looks up the
 * scratch's device address and uploads the filter taps); make that first
 * call before any stream capture.  The set-up is redone when the device's
 * context has changed since (after cudaDeviceReset), so the first call after
 * a reset must also come before any capture.  All calls share the one scratch array and
 * it keeps the previous call's contents (every level writes the LL values it
 * later reads, so nothing needs clearing); calls whose work overlaps on the
 * GPU (different streams, or different threads) race on it and must be
 * ordered by the caller.
 * Errors: EINVAL (NULL or host arrays, arrays of another device, x and u
 * overlapping, bad shape, scratch too small), ECUDA. */
MUFFIN_API muffin_status muffin_op_analysis_noalloc(const float *x, float *u,
                                                    int32_t n, int32_t nbands,
                                                    int32_t n_wavelets,
                                                    int32_t levels, void *stream);

/* ---- per-kernel profile --------------------------------------------------
 * With profiling on, every kernel the plan launches is bracketed by CUDA
 * events on the plan's stream; stats accumulate per kernel kind until the
 * next muffin_profile_enable(plan, 1).  bytes/flops are the algorithmic
 * (minimum) traffic and arithmetic of one launch. */
typedef struct {
  char name[40];
  int64_t launches;
  double total_ms;
  double bytes_per_launch;
  double flops_per_launch;
} muffin_kernel_stat;

/* on = 1 enables and clears the stats, 0 disables. */
MUFFIN_API muffin_status muffin_profile_enable(muffin_plan plan, int32_t on);
/* Copies up to capacity stats; *count = number of kernel kinds recorded. */
MUFFIN_API muffin_status muffin_profile_read(muffin_plan plan,
                                             muffin_kernel_stat *out,
                                             int32_t capacity, int32_t *count);

/* ---- host-only tables (no GPU needed) -----------------------------------
 * The FP64 tables the kernels are built from, for inspection and tests. */
/* h[0 .. 2p-1]: db<p> scaling filter by spectral factorisation, 1 <= p <= 8. */
MUFFIN_API muffin_status muffin_filter_taps(int32_t p, double *h);
/* C[k*L + l]: orthonormal DCT-II matrix, L >= 1. */
MUFFIN_API muffin_status muffin_dct_table(int32_t L, double *C);

/* Thread-local description of the last error (never NULL). */
MUFFIN_API const char *muffin_last_error(void);

/* Library version string. */
MUFFIN_API const char *muffin_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MUFFIN_H */
