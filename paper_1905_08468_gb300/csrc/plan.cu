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
// All B cubes of a plan advance in the same launches.  ADA-PT runs the group
// on y and the group on y_bar = y + eps delta per iteration; at the end of
// every window a gradient of the y-primal, one FP64 statistics pass and a
// per-cube theta update run on the device.  Repeated fixed-shape launch
// sequences (two plain iterations, one ADA-PT window) are captured once into
// CUDA graphs on the plan's own stream and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "host_math.h"
#include "kernels.h"
#include "plan_internal.h"

using namespace muffin;

namespace {

thread_local std::string g_err = "no error";

// reduction scratch layout (doubles): [0] result, [16, 16+1024) max partials;
// band sums use [0, 65 Lt); ADA-PT partials start at kRedSure + 65 Lt.
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

#define CK MUFFIN_CK

namespace muffin {

muffin_status fail(muffin_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

int set_last_error_code(int s, const char *msg) {
  g_err = msg ? msg : "";
  return s;
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace muffin

muffin_plan_s::~muffin_plan_s() {
  for (auto &kv : gplain) cudaGraphExecDestroy(kv.second);
  for (int i = 0; i < 2; ++i)
    if (gsure[i]) cudaGraphExecDestroy(gsure[i]);
  for (void *q : allocs) cudaFree(q);
  if (ev_in) cudaEventDestroy(ev_in);
  if (ev_out) cudaEventDestroy(ev_out);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (ws2) cudaStreamDestroy(ws2);
  if (ws) cudaStreamDestroy(ws);
}

namespace {

muffin_status validate(const muffin_params *p) {
  if (!p) return fail(MUFFIN_EINVAL, "params is NULL");
  if (p->n < 2 || p->n > 2048 || (p->n & (p->n - 1)))
    return fail(MUFFIN_EINVAL, "n=%d must be a power of two in [2, 2048]", p->n);
  if (p->nbands < 1 || p->nbands > 4096)
    return fail(MUFFIN_EINVAL, "nbands=%d out of range [1, 4096]", p->nbands);
  if (p->batch < 1 || (long long)p->batch * p->nbands > 65535)
    return fail(MUFFIN_EINVAL, "batch=%d must be >= 1 with batch * nbands <= 65535", p->batch);
  if (p->n_wavelets < 1 || p->n_wavelets > 8)
    return fail(MUFFIN_EINVAL, "n_wavelets=%d out of range [1, 8]", p->n_wavelets);
  if (p->levels < 0 || p->levels > 15 || (1 << p->levels) > p->n)
    return fail(MUFFIN_EINVAL, "levels=%d needs 2^levels <= n", p->levels);
  if (p->dictionary != 0 && p->dictionary != 1)
    return fail(MUFFIN_EINVAL, "dictionary=%d must be 0 (Daubechies) or 1 (IUWT)", p->dictionary);
  if (p->dictionary == 1 && p->levels > 4)
    return fail(MUFFIN_EINVAL, "the IUWT supports levels <= 4 (got %d)", p->levels);
  if (!(p->sigma > 0)) return fail(MUFFIN_EINVAL, "sigma must be > 0");
  if (!(p->tau_safety > 0 && p->tau_safety < 1))
    return fail(MUFFIN_EINVAL, "tau_safety must be in (0, 1)");
  if (p->step_rule != 0 && p->step_rule != 1)
    return fail(MUFFIN_EINVAL, "step_rule must be 0 or 1");
  if (p->precision != 0 && p->precision != 1)
    return fail(MUFFIN_EINVAL, "precision=%d must be 0 (3xTF32) or 1 (FP32)", p->precision);
  if (p->precision == 1 &&
      (p->nbands < 2 || p->nbands > 1024 || (p->nbands & (p->nbands - 1))))
    return fail(MUFFIN_EINVAL, "the FP32 spectral step needs nbands a power of two in "
                "[2, 1024] (got %d)", p->nbands);
  if (!(p->tau >= 0) || !std::isfinite(p->tau))
    return fail(MUFFIN_EINVAL, "tau must be finite and >= 0 (0: from the step rule)");
  // the spectral tile kernel keeps two [C][Lp][24] float tiles in shared memory
  const size_t lp = (size_t)(p->nbands + 15) / 16 * 16;
  if (p->precision == 0 && (size_t)2 * (p->sure ? 3 : 1) * lp * 24 * sizeof(float) > 200 * 1024)
    return fail(MUFFIN_EINVAL, "nbands=%d too large for the spectral tile (sure=%d)",
                p->nbands, p->sure);
  return MUFFIN_OK;
}

// copy a caller array (host or device) into dst (device), count floats
muffin_status fetch(muffin_plan P, const float *src, float *dst, size_t count) {
  const cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice
                                              : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(dst, src, count * sizeof(float), k, P->ws));
  return MUFFIN_OK;
}

muffin_status store(muffin_plan P, const float *src, float *dst, size_t count) {
  const cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice
                                              : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(dst, src, count * sizeof(float), k, P->ws));
  return MUFFIN_OK;
}

// NaN/Inf scan of an input already copied to the device (nimg images of N
// pixels); synchronises the work stream
muffin_status scan_input(muffin_plan P, const float *d, int nimg, const char *what) {
  double *o = P->mon + 54 * (size_t)P->Lt;
  CK(mon_state(d, nullptr, nimg, P->N, P->mon, o, P->ws));
  std::vector<double> h(3 * (size_t)nimg);
  CK(cudaMemcpyAsync(h.data(), o, h.size() * sizeof(double), cudaMemcpyDeviceToHost, P->ws));
  CK(cudaStreamSynchronize(P->ws));
  double bad = 0;
  for (int l = 0; l < nimg; ++l) bad += h[3 * (size_t)l + 2];
  if (bad > 0) return fail(MUFFIN_ENUMERIC, "%s has %.0f NaN/Inf entries", what, bad);
  return MUFFIN_OK;
}

// H^T y (unnormalised, FP64) for `nimg` bands of y already on the device
muffin_status adjoint_fp64(muffin_plan P, const float *y_dev, const double2 *hh,
                           int nimg, double2 *w, double2 *tmp) {
  const size_t cnt = (size_t)nimg * P->N;
  CK(real_to_c64(y_dev, w, cnt, P->ws));
  CK(fft2d_c64(w, tmp, P->n, nimg, false, P->tw64, P->ws));
  CK(mul_conj_c64(w, hh, cnt, P->ws));
  CK(fft2d_c64(w, tmp, P->n, nimg, true, P->tw64, P->ws));
  return MUFFIN_OK;
}

// the kernels of one iteration of group g without the x / x~ swap; a plain
// group (C = 1) may be restricted to the cubes [c0, c1)
muffin_status iterate_kernels(muffin_plan P, const Group &g, int c0, int c1,
                              cudaStream_t st = nullptr, float2 *S = nullptr,
                              float *ll = nullptr) {
  if (c1 < 0) c1 = P->B;
  if (!st) { st = P->ws; S = P->S; ll = P->llscr; }
  const int Lv = (c1 - c0) * P->L;
  Group h = g;
  WaveArgs w = P->wave(g.C);
  DctArgs d = P->dct(g.C);
  const float *kspec = P->kspec;
  if (c0 > 0) {            // only plain groups (the chain stride is the plan's)
    const size_t ov = (size_t)c0 * P->NLc;
    h.x += ov; h.xt += ov; h.v += ov; h.t += ov; h.g += ov; h.b += ov;
    h.u += ov * P->K;
    kspec += (size_t)c0 * P->L * (P->n / 2 + 1) * P->n;
    w.beta += (size_t)c0 * P->L;
    w.sc += c0;
    d.alpha += (size_t)c0 * P->N;
    d.sc += c0;
  }
  CK(launch_gradient(h.x, h.g, h.b, S, kspec, P->tw(), P->n, Lv, g.C, st,
                     P->pp(), P->grad_chunk, P->fft_radix));
  w.L = Lv;
  w.scratch = ll;
  CK(wavelet_synthesis_prox(w, h, P->p.positivity, st));
  CK(wavelet_analysis_dual(w, h, st));
  d.B = c1 - c0;
  CK(dct_dual(d, h, st));
  return MUFFIN_OK;
}

// one iteration of every chain group: with ADA-PT the two groups (on y and
// on y_bar) are independent within an iteration, so their kernels run either
// group after group (group_order 0) or phase by phase (1: both gradients,
// both syntheses, both analyses, both spectral steps).  The scratch (FFT
// spectra, LL approximations) is consumed within each call, so both orders
// compute identical results.
muffin_status iterate_groups(muffin_plan P);

// one iteration of group g; a plain group (C = 1) may be restricted to some
// runs [c0, c1) of cubes (the serving pools skip their free slots)
muffin_status iterate_group(muffin_plan P, Group &g,
                            const std::vector<std::pair<int, int>> &runs = {}) {
  if (runs.empty()) {
    muffin_status s = iterate_kernels(P, g, 0, P->B);
    if (s != MUFFIN_OK) return s;
  }
  for (const auto &r : runs) {
    muffin_status s = iterate_kernels(P, g, r.first, r.second);
    if (s != MUFFIN_OK) return s;
  }
  float *t = g.x; g.x = g.xt; g.xt = t;
  return MUFFIN_OK;
}

muffin_status iterate_groups(muffin_plan P) {
  if (P->p.sure && P->group_order == 2) {
    // the group on y_bar on the second stream with its own scratch, forked
    // from and joined back into the work stream (captured graphs keep both)
    CK(cudaEventRecord(P->ev_fork, P->ws));
    CK(cudaStreamWaitEvent(P->ws2, P->ev_fork, 0));
    muffin_status s = iterate_kernels(P, P->grp[1], 0, P->B, P->ws2, P->S2, P->llscr2);
    if (s == MUFFIN_OK) s = iterate_kernels(P, P->grp[0], 0, P->B);
    if (s != MUFFIN_OK) return s;
    CK(cudaEventRecord(P->ev_join, P->ws2));
    CK(cudaStreamWaitEvent(P->ws, P->ev_join, 0));
    for (Group *g : {&P->grp[0], &P->grp[1]}) std::swap(g->x, g->xt);
    return MUFFIN_OK;
  }
  if (!P->p.sure || P->group_order == 0) {
    muffin_status s = iterate_group(P, P->grp[0]);
    if (s == MUFFIN_OK && P->p.sure) s = iterate_group(P, P->grp[1]);
    return s;
  }
  Group *gs[2] = {&P->grp[0], &P->grp[1]};
  for (Group *g : gs)
    CK(launch_gradient(g->x, g->g, g->b, P->S, P->kspec, P->tw(), P->n, P->Lt, g->C, P->ws,
                       P->pp(), P->grad_chunk, P->fft_radix));
  for (Group *g : gs) CK(wavelet_synthesis_prox(P->wave(g->C), *g, P->p.positivity, P->ws));
  for (Group *g : gs) CK(wavelet_analysis_dual(P->wave(g->C), *g, P->ws));
  for (Group *g : gs) {
    CK(dct_dual(P->dct(g->C), *g, P->ws));
    std::swap(g->x, g->xt);
  }
  return MUFFIN_OK;
}

// zero the derivative chains (1, 2) of a C = 3 group
muffin_status reset_derivs(muffin_plan P, Group &g) {
  const size_t d = 2 * P->NL;
  CK(cudaMemsetAsync(g.x + P->NL, 0, d * sizeof(float), P->ws));
  CK(cudaMemsetAsync(g.u + P->NL * P->K, 0, d * P->K * sizeof(float), P->ws));
  CK(cudaMemsetAsync(g.v + P->NL, 0, d * sizeof(float), P->ws));
  CK(cudaMemsetAsync(g.t + P->NL, 0, d * sizeof(float), P->ws));
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

muffin_status upload_cube_const(muffin_plan P) {
  std::vector<double> cc(4 * (size_t)P->B);
  for (int c = 0; c < P->B; ++c) {
    cc[4 * c] = P->psc[c];
    cc[4 * c + 1] = P->lips[c];
    cc[4 * c + 2] = P->p.step_rule == 0 ? P->Bsum[c] : P->Bmax2[c];
    cc[4 * c + 3] = P->p.step_rule == 0 ? P->Asum[c] : P->Amax2[c];
  }
  CK(cudaMemcpyAsync(P->cube_const, cc.data(), cc.size() * sizeof(double),
                     cudaMemcpyHostToDevice, P->ws));
  CK(cudaStreamSynchronize(P->ws));
  return MUFFIN_OK;
}

// validate and install pixel weights a [B][N] and band weights bw [B][L]
// (Eq. 2regpar); the sums of their squares enter the step condition
muffin_status set_weights(muffin_plan P, const std::vector<float> &a,
                          const std::vector<float> &bw) {
  const int B = P->B, L = P->L;
  const size_t N = P->N;
  std::vector<double> as(B, 0), am(B, 0), bs(B, 0), bm(B, 0);
  for (int c = 0; c < B; ++c) {
    for (size_t i = 0; i < N; ++i) {
      const double v = a[(size_t)c * N + i];
      if (!(v >= 0) || !std::isfinite(v)) return fail(MUFFIN_EINVAL, "alpha must be finite and >= 0");
      as[c] += v * v; am[c] = std::fmax(am[c], v * v);
    }
    for (int l = 0; l < L; ++l) {
      const double v = bw[(size_t)c * L + l];
      if (!(v >= 0) || !std::isfinite(v)) return fail(MUFFIN_EINVAL, "beta must be finite and >= 0");
      bs[c] += v * v; bm[c] = std::fmax(bm[c], v * v);
    }
  }
  P->Asum = as; P->Amax2 = am; P->Bsum = bs; P->Bmax2 = bm;
  P->beta_h = bw;
  CK(cudaMemcpyAsync(P->alpha, a.data(), a.size() * 4, cudaMemcpyHostToDevice, P->ws));
  CK(cudaMemcpyAsync(P->beta, bw.data(), bw.size() * 4, cudaMemcpyHostToDevice, P->ws));
  CK(cudaStreamSynchronize(P->ws));
  return MUFFIN_OK;
}

muffin_status plan_alloc_init(muffin_plan P, const float *alpha, const float *beta) {
  const int n = P->n, L = P->L, Lt = P->Lt, B = P->B;
  const size_t N = P->N, NL = P->NL;
  const int nh = n / 2 + 1;
  CK(cudaStreamCreateWithFlags(&P->ws, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming));
  CK(P->alloc(&P->hhat, NL));
  CK(P->alloc(&P->w64a, NL));
  CK(P->alloc(&P->w64b, NL));
  CK(P->alloc(&P->kspec, (size_t)Lt * nh * n));
  P->tw_len16 = fft32_table_len(n, 16);
  CK(P->alloc(&P->tw32, (size_t)P->tw_len16 + fft32_table_len(n, 8)));
  CK(P->alloc(&P->tw64, (size_t)n));
  const size_t LL2 = (size_t)P->Lp * P->Lp;
  CK(P->alloc(&P->chi, LL2));
  CK(P->alloc(&P->clo, LL2));
  CK(P->alloc(&P->cthi, LL2));
  CK(P->alloc(&P->ctlo, LL2));
  if (P->p.precision == 1) {
    P->ftw_len = dct_f32_table_len(L) - L;
    CK(P->alloc(&P->ftab, (size_t)dct_f32_table_len(L)));
  }
  CK(P->alloc(&P->alpha, (size_t)B * N));
  CK(P->alloc(&P->beta, (size_t)Lt));
  CK(P->alloc(&P->sc, (size_t)B));
  CK(P->alloc(&P->cube_const, (size_t)4 * B));
  CK(P->alloc(&P->rec_count, 1));
  CK(P->alloc(&P->kerr, 1));
  CK(cudaMemsetAsync(P->kerr, 0, sizeof(int), P->ws));
  CK(P->alloc(&P->dred, kRedSure + 65 * (size_t)Lt + 6 * (size_t)(Lt > 4096 ? Lt : 4096)));
  CK(P->alloc(&P->wband, (size_t)Lt));
  CK(P->alloc(&P->mon, monitor_scratch_doubles(Lt)));
  CK(P->alloc(&P->S, (size_t)P->Cmax * Lt * nh * n));
  size_t off = 0;
  if (P->dict == 1) {
    off = 2 * (size_t)P->Cmax * Lt * N;       // IUWT: two running images
  } else {
    for (int j = 1; j < P->J; ++j) {
      P->lvl_off[j] = off;
      const size_t h = (size_t)(n >> j);
      off += (size_t)P->Cmax * Lt * P->K * h * h;
    }
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
    // second stream and scratch: the two chain groups may run concurrently
    CK(P->alloc(&P->S2, (size_t)P->Cmax * Lt * nh * n));
    CK(P->alloc(&P->llscr2, off ? off : 1));
    CK(cudaStreamCreateWithFlags(&P->ws2, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
  }
  P->grp[0].b = P->b;
  P->grp[1].b = P->bbar;
  P->grp_x0[0] = P->grp[0].x;
  P->grp_x0[1] = P->grp[1].x;

  // ---- twiddles: FP64 e^{-2 pi i k / n}; FP32 per-stage tables of the hot FFT
  std::vector<double2> t64(n);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    const double a = -2.0 * pi * k / n;
    t64[k] = make_double2(std::cos(a), std::sin(a));
  }
  std::vector<float2> t32((size_t)P->tw_len16 + fft32_table_len(n, 8));
  fft32_tables(n, t32.data(), 16);
  fft32_tables(n, t32.data() + P->tw_len16, 8);
  CK(cudaMemcpyAsync(P->tw32, t32.data(), t32.size() * sizeof(float2), cudaMemcpyHostToDevice, P->ws));
  CK(cudaMemcpyAsync(P->tw64, t64.data(), n * sizeof(double2), cudaMemcpyHostToDevice, P->ws));

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
  CK(cudaMemcpyAsync(P->chi, hi.data(), LL2 * 4, cudaMemcpyHostToDevice, P->ws));
  CK(cudaMemcpyAsync(P->clo, lo.data(), LL2 * 4, cudaMemcpyHostToDevice, P->ws));
  CK(cudaMemcpyAsync(P->cthi, thi.data(), LL2 * 4, cudaMemcpyHostToDevice, P->ws));
  CK(cudaMemcpyAsync(P->ctlo, tlo.data(), LL2 * 4, cudaMemcpyHostToDevice, P->ws));
  std::vector<float2> ft(P->p.precision == 1 ? (size_t)dct_f32_table_len(L) : 0);
  if (P->p.precision == 1) {
    dct_f32_tables(L, ft.data());
    CK(cudaMemcpyAsync(P->ftab, ft.data(), ft.size() * sizeof(float2), cudaMemcpyHostToDevice,
                       P->ws));
  }
  CK(cudaStreamSynchronize(P->ws));

  // ---- weights (Eq. 2regpar), per cube
  std::vector<float> a((size_t)B * N, 1.f), bw((size_t)Lt, 1.f);
  if (alpha) {
    if (is_device_ptr(alpha)) CK(cudaMemcpy(a.data(), alpha, a.size() * 4, cudaMemcpyDeviceToHost));
    else std::memcpy(a.data(), alpha, a.size() * 4);
  }
  if (beta) {
    if (is_device_ptr(beta)) CK(cudaMemcpy(bw.data(), beta, bw.size() * 4, cudaMemcpyDeviceToHost));
    else std::memcpy(bw.data(), beta, bw.size() * 4);
  }
  P->lips.assign(B, 0); P->psc.assign(B, 0); P->mu.assign(B, 0); P->gamma.assign(B, 0);
  muffin_status s2 = set_weights(P, a, bw);
  if (s2 != MUFFIN_OK) return s2;
  CK(cudaMemsetAsync(P->sc, 0, (size_t)B * sizeof(DevScalars), P->ws));
  CK(cudaStreamSynchronize(P->ws));
  return MUFFIN_OK;
}

// capture `body` on the work stream into an executable graph
template <typename F>
muffin_status capture(muffin_plan P, cudaGraphExec_t *exec, F body) {
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(P->ws, cudaStreamCaptureModeThreadLocal));
  muffin_status s = body();
  cudaError_t e = cudaStreamEndCapture(P->ws, &g);
  if (s != MUFFIN_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return fail(MUFFIN_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(MUFFIN_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return MUFFIN_OK;
}

// one ADA-PT window end: SUGAR/PSURE statistics, theta update, derivative reset
muffin_status window_end(muffin_plan P, const muffin_sure_params *sp) {
  Group &g = P->grp[0];
  Group g0 = g;
  g0.C = 1;
  CK(launch_gradient(g0.x, g0.g, g0.b, P->S, P->kspec, P->tw(), P->n, P->Lt, 1, P->ws,
                     P->pp(), P->grad_chunk, P->fft_radix));
  SureStatsArgs sa{};
  sa.grad = g.g; sa.x = g.x; sa.xb = P->grp[1].x; sa.b = P->b; sa.htd = P->htd;
  sa.wband = P->wband; sa.n = P->n; sa.L = P->Lt;
  int bpb = 0;
  double *part = P->dred + kRedSure + 65 * (size_t)P->Lt;
  {
    ProfScope ps(P->pp(), "sure_stats", 9.0 * P->NL * 4.0, 12.0 * P->NL, P->ws);
    CK(sure_stats(sa, part, &bpb, P->ws));
  }
  ThetaUpdateArgs ta{};
  ta.B = P->B; ta.sc = P->sc; ta.partials = part; ta.nb_per_cube = bpb * P->L;
  ta.record = P->records; ta.rec_count = P->rec_count;
  ta.eta_mu = sp->eta_mu; ta.eta_gamma = sp->eta_gamma; ta.theta_min = sp->theta_min;
  ta.cube_const = P->cube_const; ta.safety = P->p.tau_safety; ta.K = P->wsn2;
  ta.tau_fixed = P->p.tau;
  {
    ProfScope ps(P->pp(), "theta_update", 6.0 * 8.0 * bpb * P->Lt, 0.0, P->ws);
    CK(theta_update(ta, P->ws));
  }
  if (sp->reset_each_window) {
    muffin_status s = reset_derivs(P, P->grp[0]);
    if (s != MUFFIN_OK) return s;
    s = reset_derivs(P, P->grp[1]);
    if (s != MUFFIN_OK) return s;
  }
  return MUFFIN_OK;
}

// Results of one monitor evaluation, per cube.
struct MonOut {
  std::vector<double> rel, obj;
  std::vector<long long> nonfinite;
  long long nonfinite_total = 0;
};

// FP64 monitor of a cube of iterates x (device, [B][L][n][n]) against the
// previous iterates xo (NULL: scan x only); with y (device dirty cubes) also
// the objective (Eqs. probopt, RegAll) at x with per-cube (mu, gamma):
// the residual y - H x from an FP64 convolution (the plan's FP64 spectra),
// ||W_s x_l||_1 and ||W_lambda x^n||_1 from the FP32 transforms, all sums
// in FP64.  Synchronises the work stream.
muffin_status monitor_eval(muffin_plan P, const float *x, const float *xo, const float *y,
                           const std::vector<double> &mu, const std::vector<double> &gamma,
                           MonOut &r) {
  const int Lt = P->Lt, L = P->L, B = P->B;
  const size_t N = P->N;
  double *part = P->mon;
  double *o_state = part + 48 * (size_t)Lt, *o_res = o_state + 3 * (size_t)Lt;
  double *o_u = o_res + Lt, *o_v = o_u + Lt;
  CK(mon_state(x, xo, Lt, N, part, o_state, P->ws));
  if (y) {
    muffin_status s = ensure_op_buffers(P);
    if (s != MUFFIN_OK) return s;
    CK(real_to_c64(x, P->w64a, P->NL, P->ws));
    CK(fft2d_c64(P->w64a, P->w64b, P->n, Lt, false, P->tw64, P->ws));
    CK(mul_c64(P->w64a, P->hhat, P->NL, P->ws));
    CK(fft2d_c64(P->w64a, P->w64b, P->n, Lt, true, P->tw64, P->ws));
    CK(mon_resid2(P->w64a, y, 1.0 / (double)N, Lt, N, part, o_res, P->ws));
    CK(wavelet_analysis_op(P->wave(1), x, P->op_out, P->ws));
    CK(mon_abs(P->op_out, Lt, (size_t)P->K * N, nullptr, L, N, part, o_u, P->ws));
    CK(dct_op(P->dct(1), x, P->op_out, 0, P->ws));
    CK(mon_abs(P->op_out, Lt, N, P->alpha, L, N, part, o_v, P->ws));
  }
  std::vector<double> h(6 * (size_t)Lt);
  CK(cudaMemcpyAsync(h.data(), o_state, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                     P->ws));
  CK(cudaStreamSynchronize(P->ws));
  const double *hs = h.data(), *hr = hs + 3 * Lt, *hu = hr + Lt, *hv = hu + Lt;
  r.rel.assign(B, 0.0);
  r.obj.assign(B, std::nan(""));
  r.nonfinite.assign(B, 0);
  r.nonfinite_total = 0;
  for (int c = 0; c < B; ++c) {
    double d2 = 0, p2 = 0, nf = 0, res = 0, l1u = 0, l1v = 0;
    for (int l = c * L; l < (c + 1) * L; ++l) {
      d2 += hs[3 * l]; p2 += hs[3 * l + 1]; nf += hs[3 * l + 2];
      res += hr[l]; l1u += (double)P->beta_h[l] * hu[l]; l1v += hv[l];
    }
    r.rel[c] = p2 > 0 ? std::sqrt(d2 / p2) : (d2 > 0 ? INFINITY : 0.0);
    r.nonfinite[c] = (long long)nf;
    r.nonfinite_total += (long long)nf;
    if (y) r.obj[c] = 0.5 * res + mu[c] * l1u + gamma[c] * l1v;
  }
  return MUFFIN_OK;
}

// a check of the primal chain on y after k iterations of the current call:
// records, numeric failure, early-exit test (every cube at or below rel_tol)
muffin_status monitor_check(muffin_plan P, int k, const std::vector<double> &mu,
                            const std::vector<double> &gamma, bool *converged,
                            muffin_info *info) {
  const Group &g = P->grp[0];
  const bool obj = P->mon_p.objective != 0;
  if (obj && !P->have_y)
    return fail(MUFFIN_ESTATE, "the monitor's objective needs the dirty cube: pass it to the call");
  MonOut r;
  muffin_status s = monitor_eval(P, g.x, g.xt, obj ? P->ydev : nullptr, mu, gamma, r);
  if (s != MUFFIN_OK) return s;
  bool conv = P->mon_p.rel_tol > 0;
  for (int c = 0; c < P->B; ++c) {
    muffin_monitor_record rec{};
    rec.k = k; rec.cube = c; rec.rel_change = r.rel[c]; rec.objective = r.obj[c];
    rec.nonfinite = r.nonfinite[c];
    P->mon_rec.push_back(rec);
    if (!(r.rel[c] <= P->mon_p.rel_tol)) conv = false;
  }
  if (info) {
    info->checks += 1;
    info->rel_change = r.rel[0];
    info->objective = r.obj[0];
  }
  if (r.nonfinite_total > 0) {
    P->have_state = P->have_sure_state = false;
    return fail(MUFFIN_ENUMERIC, "%lld NaN/Inf entries in X after %d iterations",
                r.nonfinite_total, k);
  }
  *converged = conv;
  return MUFFIN_OK;
}

// end-of-call scan of the restored cube for NaN/Inf
muffin_status final_scan(muffin_plan P, int k) {
  MonOut r;
  std::vector<double> z(P->B, 0.0);
  muffin_status s = monitor_eval(P, P->grp[0].x, nullptr, nullptr, z, z, r);
  if (s != MUFFIN_OK) return s;
  if (r.nonfinite_total > 0) {
    P->have_state = P->have_sure_state = false;
    return fail(MUFFIN_ENUMERIC, "%lld NaN/Inf entries in X after %d iterations",
                r.nonfinite_total, k);
  }
  return MUFFIN_OK;
}

void info_monitor_defaults(muffin_info *info) {
  if (!info) return;
  info->checks = 0;
  info->stopped_early = 0;
  info->rel_change = std::nan("");
  info->objective = std::nan("");
}

}  // namespace

// ---------------------------------------------------------------- internal API
namespace muffin {
namespace pi {

muffin_status enter(muffin_plan P) {
  CK(cudaEventRecord(P->ev_in, P->st));
  CK(cudaStreamWaitEvent(P->ws, P->ev_in, 0));
  return MUFFIN_OK;
}

muffin_status iterate_all(muffin_plan P) {
  return iterate_groups(P);
}

void drop_graphs_and_state(muffin_plan P) {
  for (auto &kv : P->gplain) cudaGraphExecDestroy(kv.second);
  P->gplain.clear();
  for (int i = 0; i < 2; ++i)
    if (P->gsure[i]) { cudaGraphExecDestroy(P->gsure[i]); P->gsure[i] = nullptr; }
  P->have_state = false;
  P->have_sure_state = false;
  P->k_done = 0;
}

muffin_status leave(muffin_plan P, bool sync) {
  CK(cudaEventRecord(P->ev_out, P->ws));
  CK(cudaStreamWaitEvent(P->st, P->ev_out, 0));
  if (sync) {
    CK(cudaStreamSynchronize(P->ws));
    int flag = 0;
    CK(cudaMemcpy(&flag, P->kerr, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
      CK(cudaMemset(P->kerr, 0, sizeof(int)));
      P->prof.resolve();
      return fail(MUFFIN_ETIMEOUT, "spectral kernel: a bounded tensor-core wait gave up");
    }
  }
  P->prof.resolve();
  return MUFFIN_OK;
}

muffin_status load_psf(muffin_plan P, int b0, int b1, const float *psf) {
  P->vis_b = false;
  const size_t cnt = (size_t)(b1 - b0) * P->NLc;
  const size_t off = (size_t)b0 * P->NLc;
  const int nimg = (b1 - b0) * P->L;
  muffin_status s = fetch(P, psf, P->stage_a + off, cnt);
  if (s != MUFFIN_OK) return s;
  double2 *hh = P->hhat + off;
  CK(real_to_c64(P->stage_a + off, hh, cnt, P->ws));
  CK(fft2d_c64(hh, P->w64a + off, P->n, nimg, false, P->tw64, P->ws));
  const int nh = P->n / 2 + 1;
  CK(make_kspec(hh, P->kspec + (size_t)b0 * P->L * nh * P->n, 1.0 / ((double)P->n * P->n),
                P->n, nimg, P->ws));
  for (int c = b0; c < b1; ++c) {
    CK(max_abs2_c64(P->hhat + (size_t)c * P->NLc, P->NLc, P->dred + 16, P->dred, P->ws));
    double lip = 0;
    CK(cudaMemcpyAsync(&lip, P->dred, sizeof(double), cudaMemcpyDeviceToHost, P->ws));
    CK(cudaStreamSynchronize(P->ws));
    if (!(lip > 0) || !std::isfinite(lip))
      return fail(MUFFIN_EINVAL, "PSF spectrum of cube %d is zero or not finite (beta=%g)", c, lip);
    P->lips[c] = lip;
  }
  return MUFFIN_OK;
}

muffin_status load_dirty(muffin_plan P, int b0, int b1, const float *dirty) {
  P->vis_b = false;
  const size_t cnt = (size_t)(b1 - b0) * P->NLc;
  const size_t off = (size_t)b0 * P->NLc;
  muffin_status s = fetch(P, dirty, P->stage_a + off, cnt);
  if (s == MUFFIN_OK) s = scan_input(P, P->stage_a + off, (b1 - b0) * P->L, "the dirty cube");
  if (s != MUFFIN_OK) return s;
  s = adjoint_fp64(P, P->stage_a + off, P->hhat + off, (b1 - b0) * P->L, P->w64a + off,
                   P->w64b + off);
  if (s != MUFFIN_OK) return s;
  CK(c64_real_to_f32(P->w64a + off, P->b + off, 1.0 / ((double)P->n * P->n), cnt, P->ws));
  if (P->ydev) {
    CK(cudaMemcpyAsync(P->ydev + off, P->stage_a + off, cnt * sizeof(float),
                       cudaMemcpyDeviceToDevice, P->ws));
    if (b0 == 0 && b1 == P->B) P->have_y = true;
  }
  return MUFFIN_OK;
}

muffin_status reset_cubes(muffin_plan P, int gi, int b0, int b1, const float *x0_dev) {
  Group &g = P->grp[gi];
  const size_t cnt = (size_t)(b1 - b0) * P->NLc, off = (size_t)b0 * P->NLc;
  for (int c = 0; c < g.C; ++c) {
    const size_t co = (size_t)c * P->NL + off;
    CK(cudaMemsetAsync(g.x + co, 0, cnt * sizeof(float), P->ws));
    CK(cudaMemsetAsync(g.u + co * P->K, 0, cnt * P->K * sizeof(float), P->ws));
    CK(cudaMemsetAsync(g.v + co, 0, cnt * sizeof(float), P->ws));
    CK(cudaMemsetAsync(g.t + co, 0, cnt * sizeof(float), P->ws));
  }
  if (x0_dev)
    CK(cudaMemcpyAsync(g.x + off, x0_dev, cnt * sizeof(float), cudaMemcpyDeviceToDevice, P->ws));
  return MUFFIN_OK;
}

muffin_status set_theta(muffin_plan P, int b0, int b1, const double *mu, const double *gamma) {
  std::vector<DevScalars> h(b1 - b0);
  for (int c = b0; c < b1; ++c) {
    DevScalars &d = h[c - b0];
    d.mu = mu[c - b0]; d.gamma = gamma[c - b0]; d.sigma = P->p.sigma;
    d.tau = P->tau_for(c, d.mu, d.gamma);
    P->mu[c] = d.mu; P->gamma[c] = d.gamma;
  }
  CK(cudaMemcpyAsync(P->sc + b0, h.data(), h.size() * sizeof(DevScalars),
                     cudaMemcpyHostToDevice, P->ws));
  CK(cudaStreamSynchronize(P->ws));
  return MUFFIN_OK;
}

muffin_status run_plain(muffin_plan P, int iters, const std::vector<std::pair<int, int>> &runs) {
  Group &g = P->grp[0];
  Group plain = g;
  plain.C = 1;
  muffin_status s = MUFFIN_OK;
  const bool graphs = P->use_graphs && !P->profiling;
  int k = 0;
  while (k < iters) {
    const int par = plain.x == P->grp_x0[0] ? 0 : 1;
    const std::pair<int, std::vector<std::pair<int, int>>> key(par, runs);
    auto it = P->gplain.find(key);
    if (graphs && iters - k >= 2 && it == P->gplain.end() && k > 0) {
      Group cap = plain;
      cudaGraphExec_t ex = nullptr;
      s = capture(P, &ex, [&]() -> muffin_status {
        muffin_status r = iterate_group(P, cap, runs);
        if (r == MUFFIN_OK) r = iterate_group(P, cap, runs);
        return r;
      });
      if (s != MUFFIN_OK) return s;
      it = P->gplain.emplace(key, ex).first;
    }
    if (graphs && iters - k >= 2 && it != P->gplain.end()) {
      CK(cudaGraphLaunch(it->second, P->ws));
      k += 2;      // two swaps: pointers unchanged
    } else {
      s = iterate_group(P, plain, runs);
      if (s != MUFFIN_OK) return s;
      ++k;
    }
  }
  g.x = plain.x; g.xt = plain.xt;
  return MUFFIN_OK;
}

muffin_status fetch_x(muffin_plan P, int b0, int b1, float *dst) {
  return store(P, P->grp[0].x + (size_t)b0 * P->NLc, dst, (size_t)(b1 - b0) * P->NLc);
}

size_t estimate_bytes(const muffin_params *p) {
  // mirrors plan_alloc_init (each allocation carries 16 bytes of slack)
  const size_t n = p->n, L = p->nbands, B = p->batch, Lt = B * L;
  const size_t K = p->dictionary == 1 ? (size_t)p->levels + 1 : (size_t)p->n_wavelets;
  const size_t N = n * n, NL = N * Lt, nh = n / 2 + 1, C = p->sure ? 3 : 1;
  const size_t Lp = (L + 15) / 16 * 16;
  size_t ll = 0;
  if (p->dictionary == 1) ll = 2 * C * Lt * N;
  else
    for (int j = 1; j < p->levels; ++j) ll += C * Lt * K * (n >> j) * (n >> j);
  size_t b = 3 * NL * 16 + Lt * nh * n * 4 + (size_t)(fft32_table_len((int)n, 16) + fft32_table_len((int)n, 8)) * 8 + n * 16 +
             4 * Lp * Lp * 4 + B * N * 4 + Lt * 4 + B * sizeof(DevScalars) + B * 32 + 4 + 4 +
             (kRedSure + 65 * Lt + 6 * (Lt > 4096 ? Lt : 4096)) * 8 + Lt * 8 +
             C * Lt * nh * n * 8 + (ll ? ll : 1) * 4 + 3 * NL * 4 +
             C * NL * (5 + K) * 4;
  if (p->sure) b += 3 * NL * (5 + K) * 4 + 2 * NL * 4 + C * Lt * nh * n * 8 + (ll ? ll : 1) * 4;
  b += monitor_scratch_doubles((int)Lt) * 8;
  if (p->precision == 1) b += (size_t)dct_f32_table_len((int)L) * 8 + 16;
  return b + (p->sure ? 40 : 30) * 16;   // 16 bytes of slack per allocation
}

muffin_status create(const muffin_params *p, const float *psf, const float *alpha,
                     const float *beta, void *stream, muffin_plan *out) {
  if (!out) return fail(MUFFIN_EINVAL, "out is NULL");
  *out = nullptr;
  muffin_status s = validate(p);
  if (s != MUFFIN_OK) return s;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(MUFFIN_ECUDA, "no CUDA device available");
  }
  muffin_plan P = new (std::nothrow) muffin_plan_s();
  if (!P) return fail(MUFFIN_ENOMEM, "host allocation failed");
  P->p = *p;
  P->n = p->n; P->L = p->nbands; P->J = p->levels;
  P->dict = p->dictionary;
  P->dct_tc = p->nbands == 64 && p->precision == 0 ? 1 : 0;
  P->K = P->dict == 1 ? p->levels + 1 : p->n_wavelets;
  P->wsn2 = P->dict == 1 ? iuwt_norm2(p->n, p->levels) : (double)p->n_wavelets;
  P->B = p->batch; P->Lt = P->B * P->L;
  P->Lp = (P->L + 15) / 16 * 16;
  P->Cmax = p->sure ? 3 : 1;
  P->N = (size_t)P->n * P->n;
  P->NLc = P->N * P->L;
  P->NL = P->N * P->Lt;
  P->st = static_cast<cudaStream_t>(stream);
  s = plan_alloc_init(P, alpha, beta);
  if (s == MUFFIN_OK && psf) s = load_psf(P, 0, P->B, psf);
  if (s == MUFFIN_OK) s = upload_cube_const(P);
  if (s != MUFFIN_OK) {
    if (P->ws) cudaStreamSynchronize(P->ws);
    delete P;
    return s;
  }
  *out = P;
  return MUFFIN_OK;
}

}  // namespace pi
}  // namespace muffin

// ---------------------------------------------------------------- C ABI
extern "C" {

const char *muffin_last_error(void) { return g_err.c_str(); }

const char *muffin_version(void) { return "muffin-gb300 0.2 (sm_103a)"; }

void muffin_params_default(muffin_params *p, int32_t n, int32_t nbands) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->n = n; p->nbands = nbands; p->n_wavelets = 8; p->levels = 3;
  p->sigma = 10.0; p->step_rule = 0; p->tau_safety = 0.99; p->positivity = 1;
  p->sure = 0; p->batch = 1; p->dictionary = 0;
  p->precision = 0; p->tau = 0.0;
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
  if (!psf) {
    if (out) *out = nullptr;
    return fail(MUFFIN_EINVAL, "psf is NULL");
  }
  return pi::create(p, psf, alpha, beta, stream, out);
}

void muffin_plan_destroy(muffin_plan P) {
  if (!P) return;
  cudaStreamSynchronize(P->ws);
  delete P;
}

size_t muffin_plan_device_bytes(muffin_plan P) { return P ? P->bytes : 0; }

muffin_status muffin_plan_lipschitz(muffin_plan P, double *beta) {
  if (!P || !beta) return fail(MUFFIN_EINVAL, "NULL argument");
  for (int c = 0; c < P->B; ++c) beta[c] = P->lips[c];
  return MUFFIN_OK;
}

muffin_status muffin_plan_estimate_bytes(const muffin_params *p, size_t *bytes) {
  if (!bytes) return fail(MUFFIN_EINVAL, "bytes is NULL");
  muffin_status s = validate(p);
  if (s != MUFFIN_OK) return s;
  *bytes = pi::estimate_bytes(p);
  return MUFFIN_OK;
}

muffin_status muffin_plan_load_visibilities(muffin_plan P, const float *vis,
                                            const float *weights) {
  if (!P || !vis || !weights) return fail(MUFFIN_EINVAL, "NULL argument");
  const size_t cnt = P->NL;
  const int nimg = P->Lt;
  muffin_status s = pi::enter(P);
  if (s != MUFFIN_OK) return s;
  // weights -> h_hat = sqrt(m~) (FP64), |h_hat|^2 / n^2 for the FP32 gradient, beta
  s = fetch(P, weights, P->stage_a, cnt);
  if (s != MUFFIN_OK) return s;
  CK(vis_weights(P->stage_a, P->hhat, P->stage_b, P->n, nimg, P->ws));
  s = scan_input(P, P->stage_b, nimg, "the visibility weights (negative counted as NaN)");
  if (s != MUFFIN_OK) {
    const std::string msg = muffin_last_error();
    return fail(MUFFIN_EINVAL, "%s", msg.c_str());
  }
  CK(make_kspec(P->hhat, P->kspec, 1.0 / ((double)P->n * P->n), P->n, nimg, P->ws));
  for (int c = 0; c < P->B; ++c) {
    CK(max_abs2_c64(P->hhat + (size_t)c * P->NLc, P->NLc, P->dred + 16, P->dred, P->ws));
    double lip = 0;
    CK(cudaMemcpyAsync(&lip, P->dred, sizeof(double), cudaMemcpyDeviceToHost, P->ws));
    CK(cudaStreamSynchronize(P->ws));
    if (!(lip > 0) || !std::isfinite(lip))
      return fail(MUFFIN_EINVAL, "the visibility weights of cube %d are all zero", c);
    P->lips[c] = lip;
  }
  // visibilities (re, im pairs) -> b = Re U^H D = Re(unnormalised inverse DFT of D) / n
  float *vf = reinterpret_cast<float *>(P->w64b);   // 2 cnt floats fit in cnt double2
  const cudaMemcpyKind k = is_device_ptr(vis) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(vf, vis, 2 * cnt * sizeof(float), k, P->ws));
  s = scan_input(P, vf, nimg, "the visibilities");
  if (s == MUFFIN_OK) s = scan_input(P, vf + cnt, nimg, "the visibilities");
  if (s != MUFFIN_OK) return s;
  CK(vis_to_c64(vf, P->w64a, cnt, P->ws));
  CK(fft2d_c64(P->w64a, P->w64b, P->n, nimg, true, P->tw64, P->ws));
  CK(c64_real_to_f32(P->w64a, P->b, 1.0 / (double)P->n, cnt, P->ws));
  P->have_b = true;
  P->vis_b = true;
  P->have_y = false;
  s = upload_cube_const(P);
  if (s == MUFFIN_OK) s = pi::leave(P, true);
  return s;
}

muffin_status muffin_plan_load_psf(muffin_plan P, int32_t b0, int32_t b1, const float *psf) {
  if (!P || !psf) return fail(MUFFIN_EINVAL, "NULL argument");
  if (b0 < 0 || b1 > P->B || b0 >= b1) return fail(MUFFIN_EINVAL, "cube range [%d, %d) invalid", b0, b1);
  muffin_status s = pi::enter(P);
  if (s == MUFFIN_OK) s = pi::load_psf(P, b0, b1, psf);
  if (s == MUFFIN_OK) s = upload_cube_const(P);
  if (s == MUFFIN_OK) s = pi::leave(P, true);
  return s;
}

muffin_status muffin_plan_graphs(muffin_plan P, int32_t on) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  P->use_graphs = on != 0;
  return MUFFIN_OK;
}

muffin_status muffin_solve_batch(muffin_plan P, const float *dirty, float *x,
                                 int32_t iters, const double *mu, const double *gamma,
                                 int32_t flags, muffin_info *info) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  if (!x || !mu || !gamma) return fail(MUFFIN_EINVAL, "x, mu and gamma must be non-NULL");
  if (iters < 0) return fail(MUFFIN_EINVAL, "iters must be >= 0");
  for (int c = 0; c < P->B; ++c)
    if (!(mu[c] >= 0) || !(gamma[c] >= 0) || !std::isfinite(mu[c]) || !std::isfinite(gamma[c]))
      return fail(MUFFIN_EINVAL, "mu and gamma must be finite and >= 0");
  const bool warm = flags & MUFFIN_WARM;
  if (warm && !P->have_state) return fail(MUFFIN_ESTATE, "no state to continue from");
  if (!dirty && !(P->have_b && (warm || P->vis_b)))
    return fail(MUFFIN_EINVAL, "dirty is NULL (and no visibilities are loaded)");
  muffin_status s = pi::enter(P);
  if (s != MUFFIN_OK) return s;
  if (dirty) {
    s = pi::load_dirty(P, 0, P->B, dirty);
    if (s != MUFFIN_OK) return s;
    P->have_b = true;
  }
  if (!warm) {
    s = fetch(P, x, P->stage_b, P->NL);
    if (s == MUFFIN_OK) s = scan_input(P, P->stage_b, P->Lt, "X0");
    if (s == MUFFIN_OK) s = pi::reset_cubes(P, 0, 0, P->B, P->stage_b);
    if (s != MUFFIN_OK) return s;
  }
  s = pi::set_theta(P, 0, P->B, mu, gamma);
  if (s != MUFFIN_OK) return s;
  P->have_state = true;
  P->have_sure_state = false;
  if (P->mon_p.objective && !P->have_y)
    return fail(MUFFIN_ESTATE, "the monitor's objective needs the dirty cube: pass it to the call");
  muffin_info scratch_info{};
  muffin_info *inf = info ? info : &scratch_info;
  info_monitor_defaults(inf);
  P->mon_rec.clear();
  const std::vector<double> mv(mu, mu + P->B), gv(gamma, gamma + P->B);
  const int every = P->mon_p.every;
  int done = 0;
  muffin_status numeric = MUFFIN_OK;
  while (done < iters) {
    const int seg = every > 0 ? std::min(every, iters - done) : iters - done;
    s = pi::run_plain(P, seg, {});
    if (s != MUFFIN_OK) return s;
    done += seg;
    if (every > 0 && done % every == 0) {
      bool conv = false;
      s = monitor_check(P, done, mv, gv, &conv, inf);
      if (s == MUFFIN_ENUMERIC) { numeric = s; break; }
      if (s != MUFFIN_OK) return s;
      if (conv) {
        inf->stopped_early = done < iters;
        break;
      }
    }
  }
  if (numeric == MUFFIN_OK) {
    s = final_scan(P, done);
    if (s == MUFFIN_ENUMERIC) numeric = s;
    else if (s != MUFFIN_OK) return s;
  }
  const std::string numeric_msg = numeric != MUFFIN_OK ? muffin_last_error() : "";
  s = pi::fetch_x(P, 0, P->B, x);
  if (s != MUFFIN_OK) return s;
  s = pi::leave(P, true);
  if (s != MUFFIN_OK) return s;
  inf->iters_done = done; inf->tau = P->tau_for(0, mu[0], gamma[0]);
  inf->sigma = P->p.sigma; inf->lipschitz = P->lips[0];
  inf->mu = mu[0]; inf->gamma = gamma[0]; inf->records = 0;
  if (numeric != MUFFIN_OK) return fail(numeric, "%s", numeric_msg.c_str());
  return MUFFIN_OK;
}

muffin_status muffin_solve(muffin_plan P, const float *dirty, float *x,
                           int32_t iters, double mu, double gamma,
                           int32_t flags, muffin_info *info) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  std::vector<double> m(P->B, mu), g(P->B, gamma);
  return muffin_solve_batch(P, dirty, x, iters, m.data(), g.data(), flags, info);
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
  const int B = P->B;
  if (!warm)
    for (int c = 0; c < B; ++c)
      if (!(theta[2 * c] >= 0) || !(theta[2 * c + 1] >= 0))
        return fail(MUFFIN_EINVAL, "theta must be >= 0");
  muffin_status s = pi::enter(P);
  if (s != MUFFIN_OK) return s;
  const size_t NL = P->NL;
  const double scale = 1.0 / ((double)P->n * P->n);
  if (!warm) {
    // H^T y and H^T delta in FP64; b_bar = H^T y + eps H^T delta
    s = pi::load_dirty(P, 0, B, dirty);
    if (s != MUFFIN_OK) return s;
    P->have_b = true;
    s = fetch(P, delta, P->stage_b, NL);
    if (s == MUFFIN_OK) s = scan_input(P, P->stage_b, P->Lt, "delta");
    if (s != MUFFIN_OK) return s;
    s = adjoint_fp64(P, P->stage_b, P->hhat, P->Lt, P->w64b, P->w64a);
    if (s != MUFFIN_OK) return s;
    CK(c64_real_to_f32(P->w64b, P->htd, scale, NL, P->ws));
    CK(axpy_f32(P->b, P->htd, (float)sp->eps, P->bbar, NL, P->ws));
    // per-band energies and weights
    std::vector<double> ysq(P->Lt);
    CK(band_sumsq(P->stage_a, P->Lt, P->N, P->dred, P->ws));
    CK(cudaMemcpyAsync(ysq.data(), P->dred, P->Lt * sizeof(double), cudaMemcpyDeviceToHost, P->ws));
    CK(cudaStreamSynchronize(P->ws));
    std::vector<double> w(P->Lt);
    for (int c = 0; c < B; ++c) {
      double cst = 0;
      for (int l = c * P->L; l < (c + 1) * P->L; ++l) {
        if (!(noise_var[l] >= 0)) return fail(MUFFIN_EINVAL, "noise_var must be >= 0");
        cst += ysq[l] - (double)P->N * noise_var[l];
        w[l] = 2.0 * noise_var[l] / sp->eps;
      }
      P->psc[c] = cst;
    }
    CK(cudaMemcpyAsync(P->wband, w.data(), P->Lt * sizeof(double), cudaMemcpyHostToDevice, P->ws));
    s = upload_cube_const(P);
    if (s != MUFFIN_OK) return s;
    s = fetch(P, x, P->stage_b, NL);
    if (s == MUFFIN_OK) s = scan_input(P, P->stage_b, P->Lt, "X0");
    if (s == MUFFIN_OK) s = pi::reset_cubes(P, 0, 0, B, P->stage_b);
    if (s == MUFFIN_OK) s = pi::reset_cubes(P, 1, 0, B, P->stage_b);
    if (s != MUFFIN_OK) return s;
    std::vector<double> m(B), g(B);
    for (int c = 0; c < B; ++c) { m[c] = theta[2 * c]; g[c] = theta[2 * c + 1]; }
    s = pi::set_theta(P, 0, B, m.data(), g.data());
    if (s != MUFFIN_OK) return s;
    P->k_done = 0;
    P->have_state = false;
    P->have_sure_state = true;
  }
  const int cap = sp->iters / sp->window + 1;
  if (cap > P->max_records) {
    double *r = nullptr;
    CK(P->alloc(&r, (size_t)7 * B * cap));
    P->records = r;
    P->max_records = cap;
    for (int i = 0; i < 2; ++i)   // graphs hold the old record pointer
      if (P->gsure[i]) { cudaGraphExecDestroy(P->gsure[i]); P->gsure[i] = nullptr; }
  }
  CK(cudaMemsetAsync(P->rec_count, 0, sizeof(int), P->ws));
  // cached window graphs depend on the window length and the update settings
  if (P->gsure_window != sp->window || P->gsure_reset != sp->reset_each_window ||
      P->gsure_eta[0] != sp->eta_mu || P->gsure_eta[1] != sp->eta_gamma ||
      P->gsure_tmin != sp->theta_min) {
    for (int i = 0; i < 2; ++i)
      if (P->gsure[i]) { cudaGraphExecDestroy(P->gsure[i]); P->gsure[i] = nullptr; }
    P->gsure_window = sp->window; P->gsure_reset = sp->reset_each_window;
    P->gsure_eta[0] = sp->eta_mu; P->gsure_eta[1] = sp->eta_gamma; P->gsure_tmin = sp->theta_min;
  }
  const bool graphs = P->use_graphs && !P->profiling;
  std::vector<long long> rec_k;
  if (P->mon_p.objective && !P->have_y)
    return fail(MUFFIN_ESTATE, "the monitor's objective needs the dirty cube: pass it to the call");
  muffin_info scratch_info{};
  muffin_info *inf = info ? info : &scratch_info;
  info_monitor_defaults(inf);
  P->mon_rec.clear();
  muffin_status numeric = MUFFIN_OK;
  const int every = P->mon_p.every;
  int next_check = every;
  // a check at a window end at or after every `every` iterations
  auto window_check = [&](int done, bool *stop) -> muffin_status {
    *stop = false;
    if (every <= 0 || done < next_check) return MUFFIN_OK;
    while (next_check <= done) next_check += every;
    std::vector<DevScalars> th(B);
    CK(cudaMemcpyAsync(th.data(), P->sc, B * sizeof(DevScalars), cudaMemcpyDeviceToHost, P->ws));
    CK(cudaStreamSynchronize(P->ws));
    std::vector<double> m(B), g(B);
    for (int c = 0; c < B; ++c) { m[c] = th[c].mu; g[c] = th[c].gamma; }
    bool conv = false;
    muffin_status r = monitor_check(P, done, m, g, &conv, inf);
    if (r != MUFFIN_OK) return r;
    if (conv && done < sp->iters) { inf->stopped_early = 1; *stop = true; }
    return MUFFIN_OK;
  };
  int it = 0;
  while (it < sp->iters) {
    const bool at_boundary = P->k_done % sp->window == 0;
    const int par = P->grp[0].x == P->grp_x0[0] ? 0 : 1;
    if (graphs && at_boundary && sp->iters - it >= sp->window && it > 0) {
      if (!P->gsure[par]) {
        const Group c0 = P->grp[0], c1 = P->grp[1];
        s = capture(P, &P->gsure[par], [&]() -> muffin_status {
          for (int q = 0; q < sp->window; ++q) {
            muffin_status r = iterate_groups(P);
            if (r != MUFFIN_OK) return r;
          }
          return window_end(P, sp);
        });
        // capture only records the launches: restore the pointers
        P->grp[0] = c0; P->grp[1] = c1;
        if (s != MUFFIN_OK) return s;
      }
      CK(cudaGraphLaunch(P->gsure[par], P->ws));
      if (sp->window & 1) {
        std::swap(P->grp[0].x, P->grp[0].xt);
        std::swap(P->grp[1].x, P->grp[1].xt);
      }
      it += sp->window;
      P->k_done += sp->window;
      rec_k.push_back(P->k_done);
      bool stop = false;
      s = window_check(it, &stop);
      if (s == MUFFIN_ENUMERIC) { numeric = s; break; }
      if (s != MUFFIN_OK) return s;
      if (stop) break;
      continue;
    }
    s = iterate_groups(P);
    if (s != MUFFIN_OK) return s;
    ++it;
    P->k_done++;
    if (P->k_done % sp->window == 0) {
      s = window_end(P, sp);
      if (s != MUFFIN_OK) return s;
      rec_k.push_back(P->k_done);
      bool stop = false;
      s = window_check(it, &stop);
      if (s == MUFFIN_ENUMERIC) { numeric = s; break; }
      if (s != MUFFIN_OK) return s;
      if (stop) break;
    }
  }
  if (numeric == MUFFIN_OK) {
    s = final_scan(P, it);
    if (s == MUFFIN_ENUMERIC) numeric = s;
    else if (s != MUFFIN_OK) return s;
  }
  const std::string numeric_msg = numeric != MUFFIN_OK ? muffin_last_error() : "";
  const int nrec = (int)rec_k.size();
  s = pi::fetch_x(P, 0, B, x);
  if (s != MUFFIN_OK) return s;
  std::vector<DevScalars> hs(B);
  CK(cudaMemcpyAsync(hs.data(), P->sc, B * sizeof(DevScalars), cudaMemcpyDeviceToHost, P->ws));
  std::vector<double> rec((size_t)7 * B * (nrec ? nrec : 1));
  if (nrec)
    CK(cudaMemcpyAsync(rec.data(), P->records, (size_t)7 * B * nrec * sizeof(double),
                       cudaMemcpyDeviceToHost, P->ws));
  s = pi::leave(P, true);
  if (s != MUFFIN_OK) return s;
  for (int c = 0; c < B; ++c) {
    theta[2 * c] = hs[c].mu; theta[2 * c + 1] = hs[c].gamma;
    P->mu[c] = hs[c].mu; P->gamma[c] = hs[c].gamma;
  }
  if (trace)
    for (int q = 0; q < nrec; ++q)
      for (int c = 0; c < B; ++c) {
        const double *r = &rec[((size_t)q * B + c) * 7];
        muffin_sure_record &t = trace[(size_t)c * cap + q];
        t.k = (int32_t)rec_k[q]; t.mu = r[1]; t.gamma = r[2];
        t.sugar_mu = r[3]; t.sugar_gamma = r[4]; t.psure = r[5]; t.tau = r[6];
      }
  inf->iters_done = it; inf->tau = hs[0].tau; inf->sigma = P->p.sigma;
  inf->lipschitz = P->lips[0]; inf->mu = hs[0].mu; inf->gamma = hs[0].gamma;
  inf->records = nrec;
  if (numeric != MUFFIN_OK) return fail(numeric, "%s", numeric_msg.c_str());
  for (int c = 0; c < B; ++c)
    if (!std::isfinite(theta[2 * c]) || !std::isfinite(theta[2 * c + 1])) {
      P->have_state = P->have_sure_state = false;
      return fail(MUFFIN_ENUMERIC, "theta of cube %d is not finite", c);
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

}  // extern "C"

// ---------------------------------------------------------------- checkpoints
namespace {
struct BlobHeader {
  char magic[8];
  int32_t n, L, K, J, sure, B;
  long long k_done;
  int32_t have_b, have_state, have_sure_state, dict;
};

struct Seg {
  void *p;
  size_t bytes;
};

std::vector<Seg> segments(muffin_plan P) {
  std::vector<Seg> v;
  const int ng = P->p.sure ? 2 : 1;
  for (int i = 0; i < ng; ++i) {
    Group &g = P->grp[i];
    const size_t cl = (size_t)g.C * P->NL * sizeof(float);
    v.push_back({g.x, cl});
    v.push_back({g.u, cl * P->K});
    v.push_back({g.v, cl});
    v.push_back({g.t, cl});
  }
  v.push_back({P->b, P->NL * sizeof(float)});
  if (P->p.sure) {
    v.push_back({P->bbar, P->NL * sizeof(float)});
    v.push_back({P->htd, P->NL * sizeof(float)});
  }
  v.push_back({P->sc, P->B * sizeof(DevScalars)});
  v.push_back({P->wband, P->Lt * sizeof(double)});
  return v;
}
}  // namespace

extern "C" {

// ---------------------------------------------------------------- weights
muffin_status muffin_plan_set_weights(muffin_plan P, const float *alpha, const float *beta) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  std::vector<float> a((size_t)P->B * P->N), bw((size_t)P->Lt);
  // NULL keeps the current values
  CK(cudaMemcpy(a.data(), alpha ? alpha : P->alpha, a.size() * 4,
                alpha && !is_device_ptr(alpha) ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(bw.data(), beta ? beta : P->beta, bw.size() * 4,
                beta && !is_device_ptr(beta) ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost));
  return set_weights(P, a, bw);
}

muffin_status muffin_plan_weights_from_x0(muffin_plan P, const float *x0, double eps_alpha,
                                          double eps_beta, float *alpha_out, float *beta_out) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  if (!x0) return fail(MUFFIN_EINVAL, "x0 is NULL");
  if (!(eps_alpha >= 0) || !(eps_beta >= 0) || !std::isfinite(eps_alpha) || !std::isfinite(eps_beta))
    return fail(MUFFIN_EINVAL, "eps_alpha and eps_beta must be finite and >= 0");
  muffin_status s = pi::enter(P);
  if (s != MUFFIN_OK) return s;
  const size_t N = P->N, NL = P->NL;
  s = fetch(P, x0, P->stage_a, NL);
  if (s != MUFFIN_OK) return s;
  // alpha: norm of every pixel spectrum (= ||W_lambda x^n||, orthonormal DCT)
  CK(pixel_weights(P->stage_a, P->B, P->L, N, eps_alpha, P->stage_b, P->ws));
  // beta: ||W_s x_l|| = sqrt(K) ||x_l|| for the union of K orthonormal bases
  // (or K identities); the IUWT is not a tight frame, so there the planes
  // W_s x_l are computed and summed
  double bscale = (double)P->K;
  if (P->dict == 1 && P->J > 0) {
    s = ensure_op_buffers(P);
    if (s != MUFFIN_OK) return s;
    CK(wavelet_analysis_op(P->wave(1), P->stage_a, P->op_out, P->ws));
    CK(band_sumsq(P->op_out, P->Lt, (size_t)P->K * N, P->dred, P->ws));
    bscale = 1.0;
  } else {
    CK(band_sumsq(P->stage_a, P->Lt, N, P->dred, P->ws));
  }
  std::vector<float> a((size_t)P->B * N), bw((size_t)P->Lt);
  std::vector<double> ss((size_t)P->Lt);
  CK(cudaMemcpyAsync(a.data(), P->stage_b, a.size() * 4, cudaMemcpyDeviceToHost, P->ws));
  CK(cudaMemcpyAsync(ss.data(), P->dred, ss.size() * sizeof(double), cudaMemcpyDeviceToHost, P->ws));
  CK(cudaStreamSynchronize(P->ws));
  for (int l = 0; l < P->Lt; ++l)
    bw[l] = (float)(1.0 / (std::sqrt(bscale * ss[l]) + eps_beta));
  s = set_weights(P, a, bw);
  if (s != MUFFIN_OK) return s;
  if (alpha_out) s = store(P, P->alpha, alpha_out, a.size());
  if (s == MUFFIN_OK && beta_out) s = store(P, P->beta, beta_out, bw.size());
  if (s == MUFFIN_OK) s = pi::leave(P, true);
  return s;
}

// ---------------------------------------------------------------- global descent
muffin_status muffin_sure_global(muffin_plan P, const float *dirty, const float *delta,
                                 const double *noise_var, const muffin_sure_params *sp,
                                 int32_t outer, float *x, double *theta,
                                 muffin_sure_record *trace, muffin_info *info) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  if (!P->p.sure) return fail(MUFFIN_ESTATE, "plan was created without the ADA-PT chains (sure=0)");
  if (!sp || !x || !theta) return fail(MUFFIN_EINVAL, "NULL argument");
  if (outer < 0 || sp->iters < 1) return fail(MUFFIN_EINVAL, "outer >= 0 and iters >= 1 required");
  const int B = P->B;
  const size_t NL = P->NL;
  // the initial cube, restored before every outer step
  float *x0 = nullptr;
  CK(cudaMalloc(&x0, NL * sizeof(float)));
  struct Guard { float *p; ~Guard() { cudaFree(p); } } guard{x0};
  CK(cudaMemcpy(x0, x, NL * sizeof(float), cudaMemcpyDefault));
  muffin_sure_params q = *sp;
  q.window = sp->iters;              // one window of n_c iterations, theta fixed
  q.reset_each_window = 1;
  std::vector<muffin_sure_record> rec((size_t)B * 2);
  muffin_info inf{};
  for (int i = 0; i < outer; ++i) {
    if (i > 0) CK(cudaMemcpy(x, x0, NL * sizeof(float), cudaMemcpyDefault));
    muffin_status s = muffin_sure_tune(P, dirty, delta, noise_var, &q, x, theta, rec.data(), 0, &inf);
    if (s != MUFFIN_OK) return s;
    if (trace)
      for (int c = 0; c < B; ++c) trace[(size_t)c * outer + i] = rec[(size_t)c * 2];
  }
  if (info) {
    *info = inf;
    info->iters_done = outer * sp->iters;
    info->records = outer;
  }
  return MUFFIN_OK;
}

muffin_status muffin_sure_global_auto(muffin_plan P, const float *dirty, const float *delta,
                                      const double *noise_var, const muffin_sure_params *sp,
                                      int32_t outer, int32_t check, double tol, float *x,
                                      double *theta, muffin_sure_record *trace,
                                      muffin_info *info) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  if (!P->p.sure) return fail(MUFFIN_ESTATE, "plan was created without the ADA-PT chains (sure=0)");
  if (!sp || !x || !theta) return fail(MUFFIN_EINVAL, "NULL argument");
  if (outer < 0 || sp->iters < 1 || check < 1)
    return fail(MUFFIN_EINVAL, "outer >= 0, iters >= 1 and check >= 1 required");
  if (!(tol >= 0) || !std::isfinite(tol)) return fail(MUFFIN_EINVAL, "tol must be finite and >= 0");
  if (sp->iters % check != 0)
    return fail(MUFFIN_EINVAL, "the cap iters=%d must be a multiple of check=%d", sp->iters, check);
  const int B = P->B;
  const size_t NL = P->NL;
  float *x0 = nullptr;
  CK(cudaMalloc(&x0, NL * sizeof(float)));
  struct Guard { float *p; ~Guard() { cudaFree(p); } } guard{x0};
  CK(cudaMemcpy(x0, x, NL * sizeof(float), cudaMemcpyDefault));
  // theta fixed within a step: windows of `check` with no update and the
  // derivative iterates carried, so every window end yields grad R_{0:k}
  muffin_sure_params q = *sp;
  q.window = check;
  q.reset_each_window = 0;
  q.eta_mu = 0.0;
  q.eta_gamma = 0.0;
  std::vector<muffin_sure_record> rec((size_t)B * 2);
  muffin_info inf{};
  int total = 0;
  for (int i = 0; i < outer; ++i) {
    if (i > 0) CK(cudaMemcpy(x, x0, NL * sizeof(float), cudaMemcpyDefault));
    std::vector<double> prev(B, -1.0);
    std::vector<muffin_sure_record> last(B);
    int k = 0;
    for (;;) {
      q.iters = check;
      const bool warm = k > 0;
      muffin_status s = muffin_sure_tune(P, warm ? nullptr : dirty, warm ? nullptr : delta,
                                         warm ? nullptr : noise_var, &q, x, theta, rec.data(),
                                         warm ? MUFFIN_WARM : 0, &inf);
      if (s != MUFFIN_OK) return s;
      k += q.iters;
      bool settled = k >= 2 * check && inf.records > 0;
      for (int c = 0; c < B; ++c) {
        if (inf.records > 0) last[c] = rec[(size_t)c * 2];
        const double nrm = std::hypot(last[c].sugar_mu, last[c].sugar_gamma);
        if (!(std::fabs(nrm - prev[c]) <= tol * nrm)) settled = false;
        prev[c] = nrm;
      }
      if (settled || k >= sp->iters) break;
    }
    total += k;
    for (int c = 0; c < B; ++c) {   // Eq. globalgrad
      muffin_sure_record &r = last[c];
      r.k = k;
      theta[2 * c] = std::fmax(std::fma(-sp->eta_mu, r.sugar_mu, r.mu), sp->theta_min);
      theta[2 * c + 1] = std::fmax(std::fma(-sp->eta_gamma, r.sugar_gamma, r.gamma), sp->theta_min);
      if (trace) trace[(size_t)c * outer + i] = r;
    }
  }
  if (info) {
    *info = inf;
    info->iters_done = total;
    info->records = outer;
    info->mu = theta[0];
    info->gamma = theta[1];
  }
  return MUFFIN_OK;
}

// ---------------------------------------------------------------- monitor
muffin_status muffin_plan_set_monitor(muffin_plan P, const muffin_monitor_params *mp) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  if (!mp) {
    P->mon_p = muffin_monitor_params{};
    return MUFFIN_OK;
  }
  if (mp->every < 0 || !(mp->rel_tol >= 0) || !std::isfinite(mp->rel_tol))
    return fail(MUFFIN_EINVAL, "every >= 0 and a finite rel_tol >= 0 required");
  if (mp->objective && !P->ydev) {
    float *y = nullptr;
    CK(P->alloc(&y, P->NL));
    P->ydev = y;
    P->have_y = false;
  }
  P->mon_p = *mp;
  return MUFFIN_OK;
}

muffin_status muffin_plan_monitor_read(muffin_plan P, muffin_monitor_record *out,
                                       int32_t capacity, int32_t *count) {
  if (!P || !count) return fail(MUFFIN_EINVAL, "NULL argument");
  *count = (int32_t)P->mon_rec.size();
  for (int32_t i = 0; i < *count && i < capacity && out; ++i) out[i] = P->mon_rec[i];
  return MUFFIN_OK;
}

muffin_status muffin_objective(muffin_plan P, const float *dirty, const float *x,
                               const double *mu, const double *gamma, double *f) {
  if (!P || !dirty || !x || !mu || !gamma || !f) return fail(MUFFIN_EINVAL, "NULL argument");
  for (int c = 0; c < P->B; ++c)
    if (!(mu[c] >= 0) || !(gamma[c] >= 0))
      return fail(MUFFIN_EINVAL, "mu and gamma must be >= 0");
  muffin_status s = pi::enter(P);
  if (s == MUFFIN_OK) s = fetch(P, dirty, P->stage_a, P->NL);
  if (s == MUFFIN_OK) s = fetch(P, x, P->stage_b, P->NL);
  if (s != MUFFIN_OK) return s;
  MonOut r;
  const std::vector<double> m(mu, mu + P->B), g(gamma, gamma + P->B);
  s = monitor_eval(P, P->stage_b, nullptr, P->stage_a, m, g, r);
  if (s != MUFFIN_OK) return s;
  // +inf outside the positive orthant (the indicator of Eq. probopt)
  std::vector<int> neg(P->B, 0);
  if (P->p.positivity) {
    std::vector<float> h(P->NL);
    CK(cudaMemcpyAsync(h.data(), P->stage_b, P->NL * sizeof(float), cudaMemcpyDeviceToHost, P->ws));
    CK(cudaStreamSynchronize(P->ws));
    for (int c = 0; c < P->B; ++c)
      for (size_t i = (size_t)c * P->NLc; i < (size_t)(c + 1) * P->NLc && !neg[c]; ++i)
        if (h[i] < 0.f) neg[c] = 1;
  }
  s = pi::leave(P, true);
  if (s != MUFFIN_OK) return s;
  for (int c = 0; c < P->B; ++c) f[c] = neg[c] ? INFINITY : r.obj[c];
  return MUFFIN_OK;
}

// ---------------------------------------------------------------- band-sharded iteration
muffin_status muffin_shard_spatial(muffin_plan P, const float *t, float *z, double mu,
                                   double gamma, double tau) {
  if (!P || !t || !z) return fail(MUFFIN_EINVAL, "NULL argument");
  if (P->B != 1 || P->p.sure || P->dict != 0)
    return fail(MUFFIN_EINVAL, "the sharded spatial step needs a plain single-cube Daubechies plan");
  if (!P->have_state || !P->have_b)
    return fail(MUFFIN_ESTATE, "start the plan's state first (muffin_solve with iters = 0)");
  if (!(mu >= 0) || !(gamma >= 0) || !(tau > 0) || !std::isfinite(tau))
    return fail(MUFFIN_EINVAL, "mu, gamma >= 0 and tau > 0 required");
  muffin_status s = pi::enter(P);
  if (s != MUFFIN_OK) return s;
  Group &g = P->grp[0];
  s = fetch(P, t, g.t, P->NL);
  if (s != MUFFIN_OK) return s;
  DevScalars sc{mu, gamma, tau, P->p.sigma};
  CK(cudaMemcpyAsync(P->sc, &sc, sizeof sc, cudaMemcpyHostToDevice, P->ws));
  P->mu[0] = mu; P->gamma[0] = gamma;
  Group h = g;
  h.C = 1;
  CK(launch_gradient(h.x, h.g, h.b, P->S, P->kspec, P->tw(), P->n, P->Lt, 1, P->ws, P->pp(),
                     P->grad_chunk, P->fft_radix));
  WaveArgs w = P->wave(1);
  CK(wavelet_synthesis_prox(w, h, P->p.positivity, P->ws));
  CK(wavelet_analysis_dual(w, h, P->ws));
  float *zd = is_device_ptr(z) ? z : P->stage_b;
  CK(twice_minus(h.xt, h.x, zd, P->NL, P->ws));
  if (zd != z) s = store(P, zd, z, P->NL);
  if (s != MUFFIN_OK) return s;
  std::swap(g.x, g.xt);
  P->k_done++;
  return pi::leave(P, true);
}

muffin_status muffin_shard_spectral(muffin_plan P, const float *z, float *v, float *t,
                                    int64_t p0, int64_t npix, double gamma) {
  if (!P || !z || !v || !t) return fail(MUFFIN_EINVAL, "NULL argument");
  if (P->B != 1) return fail(MUFFIN_EINVAL, "the sharded spectral step needs a single-cube plan");
  if (p0 < 0 || npix < 4 || npix % 4 != 0 || (size_t)(p0 + npix) > P->N)
    return fail(MUFFIN_EINVAL, "pixel block [%lld, %lld) must lie in the image, npix a multiple of 4",
                (long long)p0, (long long)(p0 + npix));
  if (!is_device_ptr(z) || !is_device_ptr(v) || !is_device_ptr(t))
    return fail(MUFFIN_EINVAL, "z, v and t must be device arrays");
  if ((reinterpret_cast<uintptr_t>(z) | reinterpret_cast<uintptr_t>(v) |
       reinterpret_cast<uintptr_t>(t)) & 15)
    return fail(MUFFIN_EINVAL, "z, v and t must be 16-byte aligned");
  if (!(gamma >= 0)) return fail(MUFFIN_EINVAL, "gamma must be >= 0");
  muffin_status s = pi::enter(P);
  if (s != MUFFIN_OK) return s;
  DevScalars sc{0.0, gamma, 0.0, P->p.sigma};
  CK(cudaMemcpyAsync(P->sc, &sc, sizeof sc, cudaMemcpyHostToDevice, P->ws));
  Group g{};
  g.C = 1;
  g.xt = const_cast<float *>(z);     // 2 z - z = z exactly: the kernel's 2 x~ - x
  g.x = const_cast<float *>(z);
  g.v = v;
  g.t = t;
  DctArgs d = P->dct(1);
  d.npix = (size_t)npix;
  d.alpha = P->alpha + p0;
  d.B = 1;
  CK(dct_dual(d, g, P->ws));
  return pi::leave(P, true);
}

muffin_status muffin_noise_mad(muffin_plan P, const float *dirty, double *noise_var) {
  if (!P || !dirty || !noise_var) return fail(MUFFIN_EINVAL, "NULL argument");
  muffin_status s = pi::enter(P);
  if (s == MUFFIN_OK) s = fetch(P, dirty, P->stage_a, P->NL);
  if (s == MUFFIN_OK) s = scan_input(P, P->stage_a, P->Lt, "the dirty cube");
  if (s != MUFFIN_OK) return s;
  double *med = P->mon + 57 * (size_t)P->Lt, *mad = med + P->Lt, *var = mad + P->Lt;
  CK(noise_mad(P->stage_a, P->n, P->Lt, P->stage_b, med, mad, var, P->ws));
  CK(cudaMemcpyAsync(noise_var, var, P->Lt * sizeof(double), cudaMemcpyDeviceToHost, P->ws));
  return pi::leave(P, true);
}

muffin_status muffin_state_size(muffin_plan P, size_t *bytes) {
  if (!P || !bytes) return fail(MUFFIN_EINVAL, "NULL argument");
  size_t t = sizeof(BlobHeader) + 3 * P->B * sizeof(double);
  for (const Seg &s : segments(P)) t += s.bytes;
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
  std::memcpy(h.magic, "MUFFIN2", 8);
  h.n = P->n; h.L = P->L; h.K = P->K; h.J = P->J; h.sure = P->p.sure; h.B = P->B;
  h.dict = P->dict;
  h.k_done = P->k_done;
  h.have_b = P->have_b; h.have_state = P->have_state; h.have_sure_state = P->have_sure_state;
  std::memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  for (int c = 0; c < P->B; ++c) {
    const double v[3] = {P->psc[c], P->mu[c], P->gamma[c]};
    std::memcpy(o, v, sizeof(v));
    o += sizeof(v);
  }
  s = pi::enter(P);
  if (s != MUFFIN_OK) return s;
  for (const Seg &sg : segments(P)) {
    CK(cudaMemcpyAsync(o, sg.p, sg.bytes, cudaMemcpyDeviceToHost, P->ws));
    o += sg.bytes;
  }
  return pi::leave(P, true);
}

muffin_status muffin_state_import(muffin_plan P, const void *host_buf, size_t bytes) {
  size_t need = 0;
  muffin_status s = muffin_state_size(P, &need);
  if (s != MUFFIN_OK) return s;
  if (!host_buf || bytes < need) return fail(MUFFIN_EINVAL, "buffer too small (%zu < %zu)", bytes, need);
  const char *o = static_cast<const char *>(host_buf);
  BlobHeader h;
  std::memcpy(&h, o, sizeof(h));
  if (std::memcmp(h.magic, "MUFFIN2", 8) != 0 || h.n != P->n || h.L != P->L ||
      h.K != P->K || h.J != P->J || h.sure != P->p.sure || h.B != P->B || h.dict != P->dict)
    return fail(MUFFIN_EINVAL, "state blob does not match this plan");
  o += sizeof(h);
  for (int c = 0; c < P->B; ++c) {
    double v[3];
    std::memcpy(v, o, sizeof(v));
    o += sizeof(v);
    P->psc[c] = v[0]; P->mu[c] = v[1]; P->gamma[c] = v[2];
  }
  s = pi::enter(P);
  if (s != MUFFIN_OK) return s;
  for (const Seg &sg : segments(P)) {
    CK(cudaMemcpyAsync(sg.p, o, sg.bytes, cudaMemcpyHostToDevice, P->ws));
    o += sg.bytes;
  }
  s = pi::leave(P, true);
  if (s != MUFFIN_OK) return s;
  s = upload_cube_const(P);
  if (s != MUFFIN_OK) return s;
  P->k_done = h.k_done;
  P->have_b = h.have_b; P->have_state = h.have_state; P->have_sure_state = h.have_sure_state;
  return MUFFIN_OK;
}

// ---------------------------------------------------------------- operators
muffin_status muffin_op_gradient(muffin_plan P, const float *x, const float *dirty, float *g) {
  if (!P || !x || !g) return fail(MUFFIN_EINVAL, "NULL argument");
  muffin_status s = ensure_op_buffers(P);
  if (s == MUFFIN_OK) s = pi::enter(P);
  if (s != MUFFIN_OK) return s;
  const float *bb = nullptr;
  if (dirty) {
    s = fetch(P, dirty, P->stage_a, P->NL);
    if (s == MUFFIN_OK) s = adjoint_fp64(P, P->stage_a, P->hhat, P->Lt, P->w64a, P->w64b);
    if (s != MUFFIN_OK) return s;
    CK(c64_real_to_f32(P->w64a, P->op_b, 1.0 / ((double)P->n * P->n), P->NL, P->ws));
    bb = P->op_b;
  }
  s = fetch(P, x, P->op_in, P->NL);
  if (s != MUFFIN_OK) return s;
  CK(launch_gradient(P->op_in, P->op_out, bb, P->S, P->kspec, P->tw(), P->n, P->Lt, 1, P->ws,
                     nullptr, 0, P->fft_radix));
  s = store(P, P->op_out, g, P->NL);
  if (s != MUFFIN_OK) return s;
  return pi::leave(P, true);
}

muffin_status muffin_op_analysis(muffin_plan P, const float *x, float *u) {
  if (!P || !x || !u) return fail(MUFFIN_EINVAL, "NULL argument");
  muffin_status s = ensure_op_buffers(P);
  if (s == MUFFIN_OK) s = pi::enter(P);
  if (s == MUFFIN_OK) s = fetch(P, x, P->op_in, P->NL);
  if (s != MUFFIN_OK) return s;
  CK(wavelet_analysis_op(P->wave(1), P->op_in, P->op_out, P->ws));
  s = store(P, P->op_out, u, P->NL * P->K);
  if (s != MUFFIN_OK) return s;
  return pi::leave(P, true);
}

muffin_status muffin_op_synthesis(muffin_plan P, const float *u, float *x) {
  if (!P || !x || !u) return fail(MUFFIN_EINVAL, "NULL argument");
  muffin_status s = ensure_op_buffers(P);
  if (s == MUFFIN_OK) s = pi::enter(P);
  if (s == MUFFIN_OK) s = fetch(P, u, P->op_in, P->NL * P->K);
  if (s != MUFFIN_OK) return s;
  CK(wavelet_synthesis_op(P->wave(1), P->op_in, P->op_out, P->ws));
  s = store(P, P->op_out, x, P->NL);
  if (s != MUFFIN_OK) return s;
  return pi::leave(P, true);
}

muffin_status muffin_op_dct(muffin_plan P, const float *x, float *v, int32_t inverse) {
  if (!P || !x || !v) return fail(MUFFIN_EINVAL, "NULL argument");
  muffin_status s = ensure_op_buffers(P);
  if (s == MUFFIN_OK) s = pi::enter(P);
  if (s == MUFFIN_OK) s = fetch(P, x, P->op_in, P->NL);
  if (s != MUFFIN_OK) return s;
  CK(dct_op(P->dct(1), P->op_in, P->op_out, inverse, P->ws));
  s = store(P, P->op_out, v, P->NL);
  if (s != MUFFIN_OK) return s;
  return pi::leave(P, true);
}

}  // extern "C"
