// C ABI of the MUFFIN library: plans, the per-iteration schedule of
// Algorithm 2, the ADA-PT loop of Algorithm 5, checkpoints and operators.
//
// Schedule of one iteration of a chain group (C = 1 plain, C = 3 ADA-PT):
//   1. gradient      g = H^T H x - b                 (3 FFT passes)
//   2. synthesis     levels J..2 into the LL scratch, level 1 fused with the
//                    primal prox -> x~
//   3. analysis      level 1 from (x~, x) for all K bases, levels 2..J,
//                    each fused with the spatial dual update of U
//   4. spectral      DCT tile kernel: V, T
//   5. swap x <-> x~ (pointer swap)
// ADA-PT runs the group on y and the group on y_bar = y + eps delta per
// iteration; at the end of every window a gradient of the y-primal, one FP64
// statistics pass and a one-block theta update run on the device, so the
// whole loop is launch-only (no host round trip) until the call returns.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/muffin.h"
#include "host_math.h"
#include "kernels.h"

using namespace muffin;

namespace {

thread_local std::string g_err = "no error";

muffin_status fail(muffin_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(expr)                                                              \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess)                                                    \
      return fail(e_ == cudaErrorMemoryAllocation ? MUFFIN_ENOMEM : MUFFIN_ECUDA, \
                  "%s: %s", #expr, cudaGetErrorString(e_));                   \
  } while (0)

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// reduction scratch layout (doubles): [0] result, [16, 16+1024) max partials;
// band sums use [0, 65 L); ADA-PT partials start at kRedSure + 65 L.
constexpr size_t kRedSure = 1040;

// round-to-nearest (ties away) to the 10-bit TF32 mantissa
float tf32_round(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

}  // namespace

int muffin::set_last_error_code(int s, const char *msg) {
  g_err = msg ? msg : "";
  return s;
}

struct muffin_plan_s {
  muffin_params p{};
  int n = 0, L = 0, K = 0, J = 0, Lp = 0, Cmax = 1;
  size_t N = 0, NL = 0;
  cudaStream_t st = nullptr;
  std::vector<void *> allocs;
  size_t bytes = 0;

  double2 *hhat = nullptr, *w64a = nullptr, *w64b = nullptr;
  float *kspec = nullptr;
  float2 *tw32 = nullptr;
  double2 *tw64 = nullptr;
  float *chi = nullptr, *clo = nullptr, *cthi = nullptr, *ctlo = nullptr;
  float *alpha = nullptr, *beta = nullptr;
  DevScalars *sc = nullptr;
  double *dred = nullptr;      // reduction scratch
  double *wband = nullptr;     // [L]
  double *records = nullptr;   // [max_records][7]
  int max_records = 0;
  float2 *S = nullptr;
  float *llscr = nullptr;
  size_t lvl_off[16] = {};
  Group grp[2];
  float *b = nullptr, *bbar = nullptr, *htd = nullptr;
  float *stage_a = nullptr, *stage_b = nullptr;   // [L][n][n] staging
  // operator buffers (allocated on first use)
  float *op_in = nullptr, *op_out = nullptr, *op_b = nullptr;

  Prof prof;
  bool profiling = false;
  Prof *pp() { return profiling ? &prof : nullptr; }

  double lipschitz = 0, Asum = 0, Bsum = 0, Amax2 = 0, Bmax2 = 0;
  double psure_const = 0;
  bool have_b = false, have_state = false, have_sure_state = false;
  long long k_done = 0;   // ADA-PT iterations done in the current run
  double cur_mu = 0, cur_gamma = 0;

  template <typename T>
  cudaError_t alloc(T **ptr, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
    if (e != cudaSuccess) return e;
    allocs.push_back(q);
    bytes += count * sizeof(T) + 16;
    *ptr = static_cast<T *>(q);
    return cudaSuccess;
  }

  ~muffin_plan_s() {
    for (void *q : allocs) cudaFree(q);
  }

  double lnorm2(double mu, double gamma) const {
    if (p.step_rule == 0) return K * mu * mu * Bsum + gamma * gamma * Asum;
    return K * mu * mu * Bmax2 + gamma * gamma * Amax2;
  }
  double tau_for(double mu, double gamma) const {
    return p.tau_safety / (0.5 * lipschitz + p.sigma * lnorm2(mu, gamma));
  }
  WaveArgs wave() const {
    WaveArgs w{};
    w.n = n; w.L = L; w.K = K; w.J = J; w.C = Cmax;
    w.beta = beta; w.sc = sc; w.scratch = llscr;
    for (int j = 0; j < 16; ++j) w.lvl_off[j] = lvl_off[j];
    w.prof = profiling ? const_cast<Prof *>(&prof) : nullptr;
    return w;
  }
  DctArgs dct() const {
    DctArgs d{};
    d.n = n; d.L = L; d.Lp = Lp; d.C = Cmax;
    d.chi = chi; d.clo = clo; d.cthi = cthi; d.ctlo = ctlo;
    d.alpha = alpha; d.sc = sc;
    d.prof = profiling ? const_cast<Prof *>(&prof) : nullptr;
    return d;
  }
};

namespace {

muffin_status validate(const muffin_params *p) {
  if (!p) return fail(MUFFIN_EINVAL, "params is NULL");
  if (p->n < 2 || p->n > 2048 || (p->n & (p->n - 1)))
    return fail(MUFFIN_EINVAL, "n=%d must be a power of two in [2, 2048]", p->n);
  if (p->nbands < 1 || p->nbands > 4096)
    return fail(MUFFIN_EINVAL, "nbands=%d out of range [1, 4096]", p->nbands);
  if (p->n_wavelets < 1 || p->n_wavelets > 8)
    return fail(MUFFIN_EINVAL, "n_wavelets=%d out of range [1, 8]", p->n_wavelets);
  if (p->levels < 0 || p->levels > 15 || (1 << p->levels) > p->n)
    return fail(MUFFIN_EINVAL, "levels=%d needs 2^levels <= n", p->levels);
  if (!(p->sigma > 0)) return fail(MUFFIN_EINVAL, "sigma must be > 0");
  if (!(p->tau_safety > 0 && p->tau_safety < 1))
    return fail(MUFFIN_EINVAL, "tau_safety must be in (0, 1)");
  if (p->step_rule != 0 && p->step_rule != 1)
    return fail(MUFFIN_EINVAL, "step_rule must be 0 or 1");
  // the spectral tile kernel keeps two [C][Lp][24] float tiles in shared memory
  const size_t lp = (size_t)(p->nbands + 15) / 16 * 16;
  if ((size_t)2 * (p->sure ? 3 : 1) * lp * 24 * sizeof(float) > 200 * 1024)
    return fail(MUFFIN_EINVAL, "nbands=%d too large for the spectral tile (sure=%d)",
                p->nbands, p->sure);
  return MUFFIN_OK;
}

// copy a caller array (host or device) into dst (device), count floats
muffin_status fetch(muffin_plan P, const float *src, float *dst, size_t count) {
  const cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice
                                              : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(dst, src, count * sizeof(float), k, P->st));
  return MUFFIN_OK;
}

muffin_status store(muffin_plan P, const float *src, float *dst, size_t count) {
  const cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice
                                              : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(dst, src, count * sizeof(float), k, P->st));
  return MUFFIN_OK;
}

// out = (float) (H^T y) for a dirty cube y already on the device (FP64 path)
muffin_status adjoint_fp64(muffin_plan P, const float *y_dev, double2 *w,
                           double2 *tmp) {
  const size_t cnt = P->NL;
  CK(real_to_c64(y_dev, w, cnt, P->st));
  CK(fft2d_c64(w, tmp, P->n, P->L, false, P->tw64, P->st));
  CK(mul_conj_c64(w, P->hhat, cnt, P->st));
  CK(fft2d_c64(w, tmp, P->n, P->L, true, P->tw64, P->st));
  return MUFFIN_OK;
}

muffin_status set_scalars(muffin_plan P, double mu, double gamma) {
  DevScalars h{};
  h.mu = mu; h.gamma = gamma; h.sigma = P->p.sigma; h.tau = P->tau_for(mu, gamma);
  CK(cudaMemcpyAsync(P->sc, &h, sizeof(h), cudaMemcpyHostToDevice, P->st));
  CK(cudaStreamSynchronize(P->st));
  P->cur_mu = mu; P->cur_gamma = gamma;
  return MUFFIN_OK;
}

muffin_status iterate_group(muffin_plan P, Group &g) {
  CK(launch_gradient(g.x, g.g, g.b, P->S, P->kspec, P->tw32, P->n, P->L, g.C, P->st,
                     P->pp()));
  WaveArgs w = P->wave();
  w.C = g.C;
  CK(wavelet_synthesis_prox(w, g, P->p.positivity, P->st));
  CK(wavelet_analysis_dual(w, g, P->st));
  DctArgs d = P->dct();
  d.C = g.C;
  CK(dct_dual(d, g, P->st));
  float *t = g.x; g.x = g.xt; g.xt = t;
  return MUFFIN_OK;
}

muffin_status reset_group(muffin_plan P, Group &g, const float *x0_dev) {
  const size_t cl = (size_t)g.C * P->NL;
  CK(cudaMemsetAsync(g.x, 0, cl * sizeof(float), P->st));
  CK(cudaMemsetAsync(g.u, 0, cl * P->K * sizeof(float), P->st));
  CK(cudaMemsetAsync(g.v, 0, cl * sizeof(float), P->st));
  CK(cudaMemsetAsync(g.t, 0, cl * sizeof(float), P->st));
  if (x0_dev)
    CK(cudaMemcpyAsync(g.x, x0_dev, P->NL * sizeof(float), cudaMemcpyDeviceToDevice, P->st));
  return MUFFIN_OK;
}

// zero the derivative chains (1, 2) of a C = 3 group
muffin_status reset_derivs(muffin_plan P, Group &g) {
  const size_t d = 2 * P->NL;
  CK(cudaMemsetAsync(g.x + P->NL, 0, d * sizeof(float), P->st));
  CK(cudaMemsetAsync(g.u + P->NL * P->K, 0, d * P->K * sizeof(float), P->st));
  CK(cudaMemsetAsync(g.v + P->NL, 0, d * sizeof(float), P->st));
  CK(cudaMemsetAsync(g.t + P->NL, 0, d * sizeof(float), P->st));
  return MUFFIN_OK;
}

muffin_status alloc_group(muffin_plan P, Group &g, int C) {
  g.C = C;
  const size_t cl = (size_t)C * P->NL;
  CK(P->alloc(&g.x, cl));
  CK(P->alloc(&g.xt, cl));
  CK(P->alloc(&g.u, cl * P->K));
  CK(P->alloc(&g.v, cl));
  CK(P->alloc(&g.t, cl));
  CK(P->alloc(&g.g, cl));
  return MUFFIN_OK;
}

muffin_status ensure_op_buffers(muffin_plan P) {
  if (P->op_in) return MUFFIN_OK;
  CK(P->alloc(&P->op_in, P->NL * P->K));
  CK(P->alloc(&P->op_out, P->NL * P->K));
  CK(P->alloc(&P->op_b, P->NL));
  return MUFFIN_OK;
}

muffin_status plan_init(muffin_plan P, const float *psf, const float *alpha,
                        const float *beta) {
  const int n = P->n, L = P->L;
  const size_t N = P->N, NL = P->NL;
  const int nh = n / 2 + 1;
  // ---- buffers
  CK(P->alloc(&P->hhat, NL));
  CK(P->alloc(&P->w64a, NL));
  CK(P->alloc(&P->w64b, NL));
  CK(P->alloc(&P->kspec, (size_t)L * nh * n));
  CK(P->alloc(&P->tw32, (size_t)fft32_table_len(n)));
  CK(P->alloc(&P->tw64, (size_t)n));
  const size_t LL2 = (size_t)P->Lp * P->Lp;
  CK(P->alloc(&P->chi, LL2));
  CK(P->alloc(&P->clo, LL2));
  CK(P->alloc(&P->cthi, LL2));
  CK(P->alloc(&P->ctlo, LL2));
  CK(P->alloc(&P->alpha, N));
  CK(P->alloc(&P->beta, (size_t)L));
  CK(P->alloc(&P->sc, 1));
  CK(P->alloc(&P->dred, (size_t)kRedSure + 65 * (size_t)L + 6 * 4096));
  CK(P->alloc(&P->wband, (size_t)L));
  CK(P->alloc(&P->S, (size_t)P->Cmax * L * nh * n));
  size_t off = 0;
  for (int j = 1; j < P->J; ++j) {
    P->lvl_off[j] = off;
    const size_t h = (size_t)(n >> j);
    off += (size_t)P->Cmax * L * P->K * h * h;
  }
  CK(P->alloc(&P->llscr, off ? off : 1));
  CK(P->alloc(&P->b, NL));
  CK(P->alloc(&P->stage_a, NL));
  CK(P->alloc(&P->stage_b, NL));
  muffin_status s = alloc_group(P, P->grp[0], P->Cmax);
  if (s != MUFFIN_OK) return s;
  if (P->p.sure) {
    s = alloc_group(P, P->grp[1], 3);
    if (s != MUFFIN_OK) return s;
    CK(P->alloc(&P->bbar, NL));
    CK(P->alloc(&P->htd, NL));
  }
  P->grp[0].b = P->b;
  P->grp[1].b = P->bbar;

  // ---- twiddles: FP64 e^{-2 pi i k / n}; FP32 per-stage tables of the hot FFT
  std::vector<double2> t64(n);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    const double a = -2.0 * pi * k / n;
    t64[k] = make_double2(std::cos(a), std::sin(a));
  }
  std::vector<float2> t32(fft32_table_len(n));
  fft32_tables(n, t32.data());
  CK(cudaMemcpyAsync(P->tw32, t32.data(), t32.size() * sizeof(float2), cudaMemcpyHostToDevice, P->st));
  CK(cudaMemcpyAsync(P->tw64, t64.data(), n * sizeof(double2), cudaMemcpyHostToDevice, P->st));

  // ---- filters
  double taps[8][16];
  std::memset(taps, 0, sizeof(taps));
  for (int p = 1; p <= 8; ++p) daubechies_lowpass(p, taps[p - 1]);
  CK(upload_filters(taps));

  // ---- DCT tables, TF32 hi/lo split, zero padded to Lp
  std::vector<double> C((size_t)L * L);
  dct2_matrix(L, C.data());
  const int Lp = P->Lp;
  std::vector<float> hi(LL2, 0.f), lo(LL2, 0.f), thi(LL2, 0.f), tlo(LL2, 0.f);
  for (int k = 0; k < L; ++k)
    for (int l = 0; l < L; ++l) {
      const float c = (float)C[(size_t)k * L + l];
      const float h = tf32_round(c), r = tf32_round(c - h);
      hi[(size_t)k * Lp + l] = h; lo[(size_t)k * Lp + l] = r;
      thi[(size_t)l * Lp + k] = h; tlo[(size_t)l * Lp + k] = r;
    }
  CK(cudaMemcpyAsync(P->chi, hi.data(), LL2 * 4, cudaMemcpyHostToDevice, P->st));
  CK(cudaMemcpyAsync(P->clo, lo.data(), LL2 * 4, cudaMemcpyHostToDevice, P->st));
  CK(cudaMemcpyAsync(P->cthi, thi.data(), LL2 * 4, cudaMemcpyHostToDevice, P->st));
  CK(cudaMemcpyAsync(P->ctlo, tlo.data(), LL2 * 4, cudaMemcpyHostToDevice, P->st));
  CK(cudaStreamSynchronize(P->st));

  // ---- weights (Eq. 2regpar)
  std::vector<float> a(N, 1.f), bw(L, 1.f);
  if (alpha) {
    if (is_device_ptr(alpha)) CK(cudaMemcpy(a.data(), alpha, N * 4, cudaMemcpyDeviceToHost));
    else std::memcpy(a.data(), alpha, N * 4);
  }
  if (beta) {
    if (is_device_ptr(beta)) CK(cudaMemcpy(bw.data(), beta, L * 4, cudaMemcpyDeviceToHost));
    else std::memcpy(bw.data(), beta, L * 4);
  }
  P->Asum = P->Bsum = P->Amax2 = P->Bmax2 = 0;
  for (size_t i = 0; i < N; ++i) {
    const double v = a[i];
    if (!(v >= 0) || !std::isfinite(v)) return fail(MUFFIN_EINVAL, "alpha must be finite and >= 0");
    P->Asum += v * v; P->Amax2 = std::fmax(P->Amax2, v * v);
  }
  for (int l = 0; l < L; ++l) {
    const double v = bw[l];
    if (!(v >= 0) || !std::isfinite(v)) return fail(MUFFIN_EINVAL, "beta must be finite and >= 0");
    P->Bsum += v * v; P->Bmax2 = std::fmax(P->Bmax2, v * v);
  }
  CK(cudaMemcpyAsync(P->alpha, a.data(), N * 4, cudaMemcpyHostToDevice, P->st));
  CK(cudaMemcpyAsync(P->beta, bw.data(), L * 4, cudaMemcpyHostToDevice, P->st));

  // ---- PSF spectra (FP64), |h_hat|^2 / n^2 for the FP32 gradient, beta
  s = fetch(P, psf, P->stage_a, NL);
  if (s != MUFFIN_OK) return s;
  CK(real_to_c64(P->stage_a, P->hhat, NL, P->st));
  CK(fft2d_c64(P->hhat, P->w64a, n, L, false, P->tw64, P->st));
  CK(make_kspec(P->hhat, P->kspec, 1.0 / ((double)n * n), n, L, P->st));
  CK(max_abs2_c64(P->hhat, NL, P->dred + 16, P->dred, P->st));
  CK(cudaMemcpyAsync(&P->lipschitz, P->dred, sizeof(double), cudaMemcpyDeviceToHost, P->st));
  CK(cudaStreamSynchronize(P->st));
  if (!(P->lipschitz > 0) || !std::isfinite(P->lipschitz))
    return fail(MUFFIN_EINVAL, "PSF spectrum is zero or not finite (beta=%g)", P->lipschitz);
  return MUFFIN_OK;
}

muffin_status set_dirty(muffin_plan P, const float *dirty) {
  muffin_status s = fetch(P, dirty, P->stage_a, P->NL);
  if (s != MUFFIN_OK) return s;
  s = adjoint_fp64(P, P->stage_a, P->w64a, P->w64b);
  if (s != MUFFIN_OK) return s;
  CK(c64_real_to_f32(P->w64a, P->b, 1.0 / ((double)P->n * P->n), P->NL, P->st));
  P->have_b = true;
  return MUFFIN_OK;
}

}  // namespace

extern "C" {

const char *muffin_last_error(void) { return g_err.c_str(); }

const char *muffin_version(void) { return "muffin-gb300 0.1 (sm_103a)"; }

void muffin_params_default(muffin_params *p, int32_t n, int32_t nbands) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->n = n; p->nbands = nbands; p->n_wavelets = 8; p->levels = 3;
  p->sigma = 10.0; p->step_rule = 0; p->tau_safety = 0.99; p->positivity = 1;
  p->sure = 0;
}

void muffin_sure_params_default(muffin_sure_params *s) {
  if (!s) return;
  std::memset(s, 0, sizeof(*s));
  s->iters = 300; s->window = 10; s->eta_mu = 1e-3; s->eta_gamma = 1e-3;
  s->theta_min = 1e-8; s->reset_each_window = 1; s->eps = 0.0;
}

muffin_status muffin_filter_taps(int32_t p, double *h) {
  if (p < 1 || p > 8 || !h) return fail(MUFFIN_EINVAL, "p must be in [1, 8], h non-NULL");
  daubechies_lowpass(p, h);
  return MUFFIN_OK;
}

muffin_status muffin_dct_table(int32_t L, double *C) {
  if (L < 1 || !C) return fail(MUFFIN_EINVAL, "L >= 1 and C non-NULL required");
  dct2_matrix(L, C);
  return MUFFIN_OK;
}

muffin_status muffin_plan_create(const muffin_params *p, const float *psf,
                                 const float *alpha, const float *beta,
                                 void *stream, muffin_plan *out) {
  if (!out) return fail(MUFFIN_EINVAL, "out is NULL");
  *out = nullptr;
  muffin_status s = validate(p);
  if (s != MUFFIN_OK) return s;
  if (!psf) return fail(MUFFIN_EINVAL, "psf is NULL");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(MUFFIN_ECUDA, "no CUDA device available");
  }
  muffin_plan P = new (std::nothrow) muffin_plan_s();
  if (!P) return fail(MUFFIN_ENOMEM, "host allocation failed");
  P->p = *p;
  P->n = p->n; P->L = p->nbands; P->K = p->n_wavelets; P->J = p->levels;
  P->Lp = (P->L + 15) / 16 * 16;
  P->Cmax = p->sure ? 3 : 1;
  P->N = (size_t)P->n * P->n;
  P->NL = P->N * P->L;
  P->st = static_cast<cudaStream_t>(stream);
  s = plan_init(P, psf, alpha, beta);
  if (s != MUFFIN_OK) {
    delete P;
    return s;
  }
  *out = P;
  return MUFFIN_OK;
}

void muffin_plan_destroy(muffin_plan P) {
  if (!P) return;
  cudaStreamSynchronize(P->st);
  delete P;
}

size_t muffin_plan_device_bytes(muffin_plan P) { return P ? P->bytes : 0; }

muffin_status muffin_plan_lipschitz(muffin_plan P, double *beta) {
  if (!P || !beta) return fail(MUFFIN_EINVAL, "NULL argument");
  *beta = P->lipschitz;
  return MUFFIN_OK;
}

muffin_status muffin_solve(muffin_plan P, const float *dirty, float *x,
                           int32_t iters, double mu, double gamma,
                           int32_t flags, muffin_info *info) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  if (!x) return fail(MUFFIN_EINVAL, "x is NULL");
  if (iters < 0) return fail(MUFFIN_EINVAL, "iters must be >= 0");
  if (!(mu >= 0) || !(gamma >= 0) || !std::isfinite(mu) || !std::isfinite(gamma))
    return fail(MUFFIN_EINVAL, "mu and gamma must be finite and >= 0");
  const bool warm = flags & MUFFIN_WARM;
  if (warm && !P->have_state) return fail(MUFFIN_ESTATE, "no state to continue from");
  if (!dirty && !(warm && P->have_b)) return fail(MUFFIN_EINVAL, "dirty is NULL");
  muffin_status s;
  if (dirty) { s = set_dirty(P, dirty); if (s != MUFFIN_OK) return s; }
  Group &g = P->grp[0];
  Group plain = g;
  plain.C = 1;
  if (!warm) {
    s = fetch(P, x, P->stage_b, P->NL);
    if (s != MUFFIN_OK) return s;
    s = reset_group(P, plain, P->stage_b);
    if (s != MUFFIN_OK) return s;
  }
  s = set_scalars(P, mu, gamma);
  if (s != MUFFIN_OK) return s;
  P->have_state = true;
  P->have_sure_state = false;
  for (int k = 0; k < iters; ++k) {
    s = iterate_group(P, plain);
    if (s != MUFFIN_OK) return s;
  }
  // keep the swapped pointers (x <-> x~) in the plan's group
  g.x = plain.x; g.xt = plain.xt;
  s = store(P, g.x, x, P->NL);
  if (s != MUFFIN_OK) return s;
  CK(cudaStreamSynchronize(P->st));
  P->prof.resolve();
  if (info) {
    info->iters_done = iters; info->tau = P->tau_for(mu, gamma); info->sigma = P->p.sigma;
    info->lipschitz = P->lipschitz; info->mu = mu; info->gamma = gamma;
    info->records = 0;
  }
  return MUFFIN_OK;
}

muffin_status muffin_sure_tune(muffin_plan P, const float *dirty,
                               const float *delta, const double *noise_var,
                               const muffin_sure_params *sp, float *x,
                               double *theta, muffin_sure_record *trace,
                               int32_t flags, muffin_info *info) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  if (!P->p.sure) return fail(MUFFIN_ESTATE, "plan was created without the ADA-PT chains (sure=0)");
  if (!sp || !x || !theta) return fail(MUFFIN_EINVAL, "NULL argument");
  if (sp->iters < 0 || sp->window < 1) return fail(MUFFIN_EINVAL, "iters >= 0 and window >= 1 required");
  if (!(sp->eps > 0)) return fail(MUFFIN_EINVAL, "eps must be > 0");
  const bool warm = flags & MUFFIN_WARM;
  if (warm && !P->have_sure_state) return fail(MUFFIN_ESTATE, "no ADA-PT state to continue from");
  if (!warm && (!dirty || !delta || !noise_var))
    return fail(MUFFIN_EINVAL, "dirty, delta and noise_var are required");
  if (!warm && (!(theta[0] >= 0) || !(theta[1] >= 0)))
    return fail(MUFFIN_EINVAL, "theta must be >= 0");
  muffin_status s;
  const size_t NL = P->NL;
  const double scale = 1.0 / ((double)P->n * P->n);
  if (!warm) {
    // H^T y and H^T delta in FP64; b_bar = H^T (y + eps delta)
    s = set_dirty(P, dirty);
    if (s != MUFFIN_OK) return s;
    s = fetch(P, delta, P->stage_b, NL);
    if (s != MUFFIN_OK) return s;
    s = adjoint_fp64(P, P->stage_b, P->w64b, P->w64a);
    if (s != MUFFIN_OK) return s;
    CK(c64_real_to_f32(P->w64b, P->htd, scale, NL, P->st));
    CK(axpy_f32(P->b, P->htd, (float)sp->eps, P->bbar, NL, P->st));
    // per-band energies and weights
    std::vector<double> ysq(P->L);
    CK(band_sumsq(P->stage_a, P->L, P->N, P->dred, P->st));
    CK(cudaMemcpyAsync(ysq.data(), P->dred, P->L * sizeof(double), cudaMemcpyDeviceToHost, P->st));
    CK(cudaStreamSynchronize(P->st));
    std::vector<double> w(P->L);
    double c = 0;
    for (int l = 0; l < P->L; ++l) {
      if (!(noise_var[l] >= 0)) return fail(MUFFIN_EINVAL, "noise_var must be >= 0");
      c += ysq[l] - (double)P->N * noise_var[l];
      w[l] = 2.0 * noise_var[l] / sp->eps;
    }
    P->psure_const = c;
    CK(cudaMemcpyAsync(P->wband, w.data(), P->L * sizeof(double), cudaMemcpyHostToDevice, P->st));
    s = fetch(P, x, P->stage_b, NL);
    if (s != MUFFIN_OK) return s;
    s = reset_group(P, P->grp[0], P->stage_b);
    if (s != MUFFIN_OK) return s;
    s = reset_group(P, P->grp[1], P->stage_b);
    if (s != MUFFIN_OK) return s;
    s = set_scalars(P, theta[0], theta[1]);
    if (s != MUFFIN_OK) return s;
    P->k_done = 0;
    P->have_state = false;
    P->have_sure_state = true;
  }
  const int nrec_max = sp->iters / sp->window + 1;
  if (nrec_max > P->max_records) {
    double *r = nullptr;
    CK(P->alloc(&r, (size_t)7 * nrec_max));
    P->records = r;
    P->max_records = nrec_max;
  }
  const double rule_B = P->p.step_rule == 0 ? P->Bsum : P->Bmax2;
  const double rule_A = P->p.step_rule == 0 ? P->Asum : P->Amax2;
  int nrec = 0;
  for (int it = 0; it < sp->iters; ++it) {
    s = iterate_group(P, P->grp[0]);
    if (s != MUFFIN_OK) return s;
    s = iterate_group(P, P->grp[1]);
    if (s != MUFFIN_OK) return s;
    P->k_done++;
    if (P->k_done % sp->window == 0) {
      Group &g = P->grp[0];
      // gradient of the y-primal at the new x (chain 0 only)
      CK(launch_gradient(g.x, g.g, g.b, P->S, P->kspec, P->tw32, P->n, P->L, 1, P->st,
                         P->pp()));
      SureStatsArgs sa{};
      sa.grad = g.g; sa.x = g.x; sa.xb = P->grp[1].x; sa.b = P->b; sa.htd = P->htd;
      sa.wband = P->wband; sa.n = P->n; sa.L = P->L;
      int nb = 0;
      double *part = P->dred + kRedSure + 65 * (size_t)P->L;
      {
        ProfScope ps(P->pp(), "sure_stats", 9.0 * NL * 4.0, 12.0 * NL, P->st);
        CK(sure_stats(sa, part, &nb, P->st));
      }
      ThetaUpdateArgs ta{};
      ta.sc = P->sc; ta.partials = part; ta.nblocks = nb;
      ta.record = P->records + 7 * nrec;
      ta.k = (int)P->k_done;
      ta.eta_mu = sp->eta_mu; ta.eta_gamma = sp->eta_gamma; ta.theta_min = sp->theta_min;
      ta.psure_const = P->psure_const;
      ta.safety = P->p.tau_safety; ta.lipschitz = P->lipschitz; ta.K = P->K;
      ta.Bsum = rule_B; ta.Asum = rule_A;
      {
        ProfScope ps(P->pp(), "theta_update", 6.0 * 8.0 * nb, 0.0, P->st);
        CK(theta_update(ta, P->st));
      }
      ++nrec;
      if (sp->reset_each_window) {
        s = reset_derivs(P, P->grp[0]);
        if (s != MUFFIN_OK) return s;
        s = reset_derivs(P, P->grp[1]);
        if (s != MUFFIN_OK) return s;
      }
    }
  }
  s = store(P, P->grp[0].x, x, NL);
  if (s != MUFFIN_OK) return s;
  DevScalars hs{};
  CK(cudaMemcpyAsync(&hs, P->sc, sizeof(hs), cudaMemcpyDeviceToHost, P->st));
  std::vector<double> rec((size_t)7 * (nrec ? nrec : 1));
  if (nrec)
    CK(cudaMemcpyAsync(rec.data(), P->records, (size_t)7 * nrec * sizeof(double),
                       cudaMemcpyDeviceToHost, P->st));
  CK(cudaStreamSynchronize(P->st));
  P->prof.resolve();
  theta[0] = hs.mu; theta[1] = hs.gamma;
  P->cur_mu = hs.mu; P->cur_gamma = hs.gamma;
  if (trace)
    for (int q = 0; q < nrec; ++q) {
      const double *r = &rec[(size_t)7 * q];
      trace[q].k = (int32_t)r[0]; trace[q].mu = r[1]; trace[q].gamma = r[2];
      trace[q].sugar_mu = r[3]; trace[q].sugar_gamma = r[4]; trace[q].psure = r[5];
      trace[q].tau = r[6];
    }
  if (info) {
    info->iters_done = sp->iters; info->tau = hs.tau; info->sigma = P->p.sigma;
    info->lipschitz = P->lipschitz; info->mu = hs.mu; info->gamma = hs.gamma;
    info->records = nrec;
  }
  return MUFFIN_OK;
}

// ---------------------------------------------------------------- profile
muffin_status muffin_profile_enable(muffin_plan P, int32_t on) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  P->prof.resolve();
  if (on) P->prof.stats.clear();
  P->profiling = on != 0;
  return MUFFIN_OK;
}

muffin_status muffin_profile_read(muffin_plan P, muffin_kernel_stat *out,
                                  int32_t capacity, int32_t *count) {
  if (!P || !count) return fail(MUFFIN_EINVAL, "NULL argument");
  P->prof.resolve();
  *count = (int32_t)P->prof.stats.size();
  for (int32_t i = 0; i < *count && i < capacity && out; ++i) {
    const Prof::Stat &st = P->prof.stats[i];
    std::memset(out[i].name, 0, sizeof(out[i].name));
    std::strncpy(out[i].name, st.name.c_str(), sizeof(out[i].name) - 1);
    out[i].launches = st.launches;
    out[i].total_ms = st.total_ms;
    out[i].bytes_per_launch = st.bytes;
    out[i].flops_per_launch = st.flops;
  }
  return MUFFIN_OK;
}

// ---------------------------------------------------------------- checkpoints
namespace {
struct BlobHeader {
  char magic[8];
  int32_t n, L, K, J, sure, pad;
  long long k_done;
  double psure_const, cur_mu, cur_gamma;
  int32_t have_b, have_state, have_sure_state, pad2;
};

struct Seg {
  float *p;
  size_t count;
};

std::vector<Seg> segments(muffin_plan P) {
  std::vector<Seg> v;
  const int ng = P->p.sure ? 2 : 1;
  for (int i = 0; i < ng; ++i) {
    Group &g = P->grp[i];
    const size_t cl = (size_t)g.C * P->NL;
    v.push_back({g.x, cl});
    v.push_back({g.u, cl * P->K});
    v.push_back({g.v, cl});
    v.push_back({g.t, cl});
  }
  v.push_back({P->b, P->NL});
  if (P->p.sure) {
    v.push_back({P->bbar, P->NL});
    v.push_back({P->htd, P->NL});
  }
  return v;
}
}  // namespace

muffin_status muffin_state_size(muffin_plan P, size_t *bytes) {
  if (!P || !bytes) return fail(MUFFIN_EINVAL, "NULL argument");
  size_t t = sizeof(BlobHeader) + sizeof(DevScalars) + P->L * sizeof(double);
  for (const Seg &s : segments(P)) t += s.count * sizeof(float);
  *bytes = t;
  return MUFFIN_OK;
}

muffin_status muffin_state_export(muffin_plan P, void *host_buf, size_t bytes) {
  size_t need = 0;
  muffin_status s = muffin_state_size(P, &need);
  if (s != MUFFIN_OK) return s;
  if (!host_buf || bytes < need) return fail(MUFFIN_EINVAL, "buffer too small (%zu < %zu)", bytes, need);
  char *o = static_cast<char *>(host_buf);
  BlobHeader h{};
  std::memcpy(h.magic, "MUFFIN1", 8);
  h.n = P->n; h.L = P->L; h.K = P->K; h.J = P->J; h.sure = P->p.sure;
  h.k_done = P->k_done; h.psure_const = P->psure_const;
  h.cur_mu = P->cur_mu; h.cur_gamma = P->cur_gamma;
  h.have_b = P->have_b; h.have_state = P->have_state; h.have_sure_state = P->have_sure_state;
  std::memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  CK(cudaMemcpyAsync(o, P->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, P->st));
  o += sizeof(DevScalars);
  CK(cudaMemcpyAsync(o, P->wband, P->L * sizeof(double), cudaMemcpyDeviceToHost, P->st));
  o += P->L * sizeof(double);
  for (const Seg &sg : segments(P)) {
    CK(cudaMemcpyAsync(o, sg.p, sg.count * sizeof(float), cudaMemcpyDeviceToHost, P->st));
    o += sg.count * sizeof(float);
  }
  CK(cudaStreamSynchronize(P->st));
  return MUFFIN_OK;
}

muffin_status muffin_state_import(muffin_plan P, const void *host_buf, size_t bytes) {
  size_t need = 0;
  muffin_status s = muffin_state_size(P, &need);
  if (s != MUFFIN_OK) return s;
  if (!host_buf || bytes < need) return fail(MUFFIN_EINVAL, "buffer too small (%zu < %zu)", bytes, need);
  const char *o = static_cast<const char *>(host_buf);
  BlobHeader h;
  std::memcpy(&h, o, sizeof(h));
  if (std::memcmp(h.magic, "MUFFIN1", 8) != 0 || h.n != P->n || h.L != P->L ||
      h.K != P->K || h.J != P->J || h.sure != P->p.sure)
    return fail(MUFFIN_EINVAL, "state blob does not match this plan");
  o += sizeof(h);
  CK(cudaMemcpyAsync(P->sc, o, sizeof(DevScalars), cudaMemcpyHostToDevice, P->st));
  o += sizeof(DevScalars);
  CK(cudaMemcpyAsync(P->wband, o, P->L * sizeof(double), cudaMemcpyHostToDevice, P->st));
  o += P->L * sizeof(double);
  for (const Seg &sg : segments(P)) {
    CK(cudaMemcpyAsync(sg.p, o, sg.count * sizeof(float), cudaMemcpyHostToDevice, P->st));
    o += sg.count * sizeof(float);
  }
  CK(cudaStreamSynchronize(P->st));
  P->k_done = h.k_done; P->psure_const = h.psure_const;
  P->cur_mu = h.cur_mu; P->cur_gamma = h.cur_gamma;
  P->have_b = h.have_b; P->have_state = h.have_state; P->have_sure_state = h.have_sure_state;
  return MUFFIN_OK;
}

// ---------------------------------------------------------------- operators
muffin_status muffin_op_gradient(muffin_plan P, const float *x, const float *dirty, float *g) {
  if (!P || !x || !g) return fail(MUFFIN_EINVAL, "NULL argument");
  muffin_status s = ensure_op_buffers(P);
  if (s != MUFFIN_OK) return s;
  const float *bb = nullptr;
  if (dirty) {
    s = fetch(P, dirty, P->stage_a, P->NL);
    if (s != MUFFIN_OK) return s;
    s = adjoint_fp64(P, P->stage_a, P->w64a, P->w64b);
    if (s != MUFFIN_OK) return s;
    CK(c64_real_to_f32(P->w64a, P->op_b, 1.0 / ((double)P->n * P->n), P->NL, P->st));
    bb = P->op_b;
  }
  s = fetch(P, x, P->op_in, P->NL);
  if (s != MUFFIN_OK) return s;
  CK(launch_gradient(P->op_in, P->op_out, bb, P->S, P->kspec, P->tw32, P->n, P->L, 1, P->st));
  s = store(P, P->op_out, g, P->NL);
  if (s != MUFFIN_OK) return s;
  CK(cudaStreamSynchronize(P->st));
  return MUFFIN_OK;
}

muffin_status muffin_op_analysis(muffin_plan P, const float *x, float *u) {
  if (!P || !x || !u) return fail(MUFFIN_EINVAL, "NULL argument");
  muffin_status s = ensure_op_buffers(P);
  if (s != MUFFIN_OK) return s;
  s = fetch(P, x, P->op_in, P->NL);
  if (s != MUFFIN_OK) return s;
  WaveArgs w = P->wave();
  w.C = 1;
  CK(wavelet_analysis_op(w, P->op_in, P->op_out, P->st));
  s = store(P, P->op_out, u, P->NL * P->K);
  if (s != MUFFIN_OK) return s;
  CK(cudaStreamSynchronize(P->st));
  return MUFFIN_OK;
}

muffin_status muffin_op_synthesis(muffin_plan P, const float *u, float *x) {
  if (!P || !x || !u) return fail(MUFFIN_EINVAL, "NULL argument");
  muffin_status s = ensure_op_buffers(P);
  if (s != MUFFIN_OK) return s;
  s = fetch(P, u, P->op_in, P->NL * P->K);
  if (s != MUFFIN_OK) return s;
  WaveArgs w = P->wave();
  w.C = 1;
  CK(wavelet_synthesis_op(w, P->op_in, P->op_out, P->st));
  s = store(P, P->op_out, x, P->NL);
  if (s != MUFFIN_OK) return s;
  CK(cudaStreamSynchronize(P->st));
  return MUFFIN_OK;
}

muffin_status muffin_op_dct(muffin_plan P, const float *x, float *v, int32_t inverse) {
  if (!P || !x || !v) return fail(MUFFIN_EINVAL, "NULL argument");
  muffin_status s = ensure_op_buffers(P);
  if (s != MUFFIN_OK) return s;
  s = fetch(P, x, P->op_in, P->NL);
  if (s != MUFFIN_OK) return s;
  DctArgs d = P->dct();
  d.C = 1;
  CK(dct_op(d, P->op_in, P->op_out, inverse, P->st));
  s = store(P, P->op_out, v, P->NL);
  if (s != MUFFIN_OK) return s;
  CK(cudaStreamSynchronize(P->st));
  return MUFFIN_OK;
}

}  // extern "C"
