// Per-shape choice of launch variants for the hot kernels (the wavelet
// synthesis row pass, the spectral kernel and its grid, the chunking of the
// gradient's FFT passes).  Every
// variant yields identical results; only speed differs, and it depends on
// the cube shape and the GPU, so the plan times the candidates on its own
// buffers and caches the winner per shape, in process and optionally in a
// text file.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "plan_internal.h"

namespace {

using muffin::fail;

struct Choice {
  int syn_packed = 0;
  int dct_ctas = 0;
  int dct_tc = 0;      // spectral step on tcgen05 (64-band plans)
  int grad_chunk = 0;  // images per pass of the gradient FFTs (0: all)
  int fft_radix = 16;  // largest radix of the gradient FFT plan
  int group_order = 0; // ADA-PT groups: 0 one after the other, 1 phase by phase, 2 two streams
  int ana_ring = 0;    // analysis U staging in a shared-memory ring
  int ana_pipe = 0;    // level-1 analysis: chain-major, one barrier per step
};

std::mutex g_mu;
std::map<std::string, Choice> g_cache;

std::string shape_key(muffin_plan P) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  std::string name(prop.name);
  for (char &ch : name)
    if (ch == ' ' || ch == '\t') ch = '_';
  char buf[256];
  std::snprintf(buf, sizeof buf,
                "n=%d,L=%d,B=%d,C=%d,J=%d,K=%d,dict=%d,sure=%d,prec=%d,sm=%d,dev=%s", P->n,
                P->L, P->B, P->Cmax, P->J, P->K, P->dict, P->p.sure ? 1 : 0, P->p.precision,
                sms, name.c_str());
  return buf;
}

// the last line "muffin-tune-6 <key> <syn_packed> <dct_ctas> <dct_tc> <grad_chunk>
// <fft_radix> <group_order> <ana_ring> <ana_pipe>" with this key
bool file_lookup(const char *path, const std::string &key, Choice *c) {
  FILE *f = std::fopen(path, "r");
  if (!f) return false;
  char line[512], tag[32], k[400];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    int a = 0, b = 0, t = 0, g = 0, r = 0, o = 0, ar = 0, ap = 0;
    if (std::sscanf(line, "%31s %399s %d %d %d %d %d %d %d %d", tag, k, &a, &b, &t, &g, &r, &o,
                    &ar, &ap) != 10)
      continue;
    if (std::strcmp(tag, "muffin-tune-6") != 0 || key != k) continue;
    if (a < 0 || a > 3 || b < 0 || t < 0 || t > 1 || g < 0 || (r != 8 && r != 16) ||
        o < 0 || o > 2 || ar < 0 || ar > 1 || ap < 0 || ap > 1)
      continue;
    c->ana_ring = ar;
    c->ana_pipe = ap;
    c->syn_packed = a;
    c->dct_ctas = b;
    c->dct_tc = t;
    c->grad_chunk = g;
    c->fft_radix = r;
    c->group_order = o;
    found = true;
  }
  std::fclose(f);
  return found;
}

void file_append(const char *path, const std::string &key, const Choice &c) {
  FILE *f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "muffin-tune-6 %s %d %d %d %d %d %d %d %d\n", key.c_str(), c.syn_packed,
               c.dct_ctas, c.dct_tc, c.grad_chunk, c.fft_radix, c.group_order, c.ana_ring,
               c.ana_pipe);
  std::fclose(f);
}

void apply(muffin_plan P, const Choice &c) {
  P->syn_packed = c.syn_packed;
  P->dct_ctas = c.dct_ctas;
  P->dct_tc = P->L == 64 && P->p.precision == 0 ? c.dct_tc : 0;
  P->grad_chunk = c.grad_chunk;
  P->fft_radix = P->n >= 64 ? c.fft_radix : 16;
  P->group_order = P->p.sure ? c.group_order : 0;
  P->ana_ring = c.ana_ring;
  P->ana_pipe = c.ana_pipe;
}

// mean time of one iteration of every chain group with choice c
muffin_status time_choice(muffin_plan P, const Choice &c, int reps, cudaEvent_t e0,
                          cudaEvent_t e1, double *ms) {
  apply(P, c);
  for (int w = 0; w < 2; ++w) {
    muffin_status s = muffin::pi::iterate_all(P);
    if (s != MUFFIN_OK) return s;
  }
  MUFFIN_CK(cudaEventRecord(e0, P->ws));
  for (int r = 0; r < reps; ++r) {
    muffin_status s = muffin::pi::iterate_all(P);
    if (s != MUFFIN_OK) return s;
  }
  MUFFIN_CK(cudaEventRecord(e1, P->ws));
  MUFFIN_CK(cudaEventSynchronize(e1));
  float t = 0.f;
  MUFFIN_CK(cudaEventElapsedTime(&t, e0, e1));
  *ms = t / reps;
  return MUFFIN_OK;
}

muffin_status tune(muffin_plan P, Choice *best, muffin_tune_info *info) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MUFFIN_CK(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(MUFFIN_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(ce));
  }
  const bool was_profiling = P->profiling;
  P->profiling = false;
  muffin_status s = muffin::pi::enter(P);
  // about 3 repetitions per candidate above a million voxels, more below
  const double vox = (double)P->NL * P->Cmax * (P->p.sure ? 2 : 1);
  const int reps = vox >= 2e7 ? 3 : (vox >= 1e6 ? 5 : 10);
  Choice cur{};
  const bool tf32 = P->p.precision == 0;   // the FP32 spectral step has no variants
  cur.dct_tc = P->L == 64 && tf32 ? 1 : 0; // the default kernel for 64 bands
  double t_def = 0.0, t_best = 0.0;
  int cand = 0;
  if (s == MUFFIN_OK) s = time_choice(P, cur, reps, e0, e1, &t_def);
  t_best = t_def;
  *best = cur;
  ++cand;
  // coordinate search: synthesis variants, then the spectral grid
  for (int v = 1; v <= 3 && s == MUFFIN_OK; ++v) {
    Choice c = *best;
    c.syn_packed = v;
    double t = 0.0;
    s = time_choice(P, c, reps, e0, e1, &t);
    ++cand;
    if (s == MUFFIN_OK && t < t_best) { t_best = t; *best = c; }
  }
  if (P->L == 64 && tf32 && s == MUFFIN_OK) {     // the other spectral kernel
    Choice c = *best;
    c.dct_tc = 0;
    double t = 0.0;
    s = time_choice(P, c, reps, e0, e1, &t);
    ++cand;
    if (s == MUFFIN_OK && t < t_best) { t_best = t; *best = c; }
  }
  for (int k = 1; k <= 2 && tf32 && s == MUFFIN_OK && !best->dct_tc; ++k) {
    Choice c = *best;
    c.dct_ctas = k;
    double t = 0.0;
    s = time_choice(P, c, reps, e0, e1, &t);
    ++cand;
    if (s == MUFFIN_OK && t < t_best) { t_best = t; *best = c; }
  }
  // the gradient's FFT passes over image chunks whose spectra fit in L2
  // (the images of one gradient call: C L of a chain group)
  const int nimg = P->Cmax * P->Lt;
  for (int q : {48, 16}) {
    if (q >= nimg || s != MUFFIN_OK) continue;
    Choice c = *best;
    c.grad_chunk = q;
    double t = 0.0;
    s = time_choice(P, c, reps, e0, e1, &t);
    ++cand;
    if (s == MUFFIN_OK && t < t_best) { t_best = t; *best = c; }
  }
  if (P->n >= 64 && s == MUFFIN_OK) {   // the radix-8 FFT plan
    Choice c = *best;
    c.fft_radix = 8;
    double t = 0.0;
    s = time_choice(P, c, reps, e0, e1, &t);
    ++cand;
    if (s == MUFFIN_OK && t < t_best) { t_best = t; *best = c; }
  }
  // the analysis U ring, where the size-specialised analysis runs
  if ((P->n == 512 || P->n == 1024 || P->n == 2048) && P->J > 1 && P->dict == 0 &&
      s == MUFFIN_OK) {
    Choice c = *best;
    c.ana_ring = 1;
    double t = 0.0;
    s = time_choice(P, c, reps, e0, e1, &t);
    ++cand;
    if (s == MUFFIN_OK && t < t_best) { t_best = t; *best = c; }
  }
  // the other level-1 analysis kernel (iterations with more than one level),
  // after the ring, so that it is timed with the ring choice in place
  if (P->J > 1 && P->dict == 0 && s == MUFFIN_OK) {
    Choice c = *best;
    c.ana_pipe = 1 - c.ana_pipe;
    double t = 0.0;
    s = time_choice(P, c, reps, e0, e1, &t);
    ++cand;
    if (s == MUFFIN_OK && t < t_best) { t_best = t; *best = c; }
  }
  for (int o = 1; o <= 2 && P->p.sure && s == MUFFIN_OK; ++o) {   // kernel order of the groups
    Choice c = *best;
    c.group_order = o;
    double t = 0.0;
    s = time_choice(P, c, reps, e0, e1, &t);
    ++cand;
    if (s == MUFFIN_OK && t < t_best) { t_best = t; *best = c; }
  }
  if (s == MUFFIN_OK) s = muffin::pi::leave(P, true);
  P->profiling = was_profiling;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != MUFFIN_OK) return s;
  if (info) {
    info->candidates = cand;
    info->ms_default = t_def;
    info->ms_best = t_best;
  }
  return MUFFIN_OK;
}

}  // namespace

extern "C" {

muffin_status muffin_plan_set_spectral_kernel(muffin_plan P, int32_t tcgen05) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  if (tcgen05 != 0 && tcgen05 != 1) return fail(MUFFIN_EINVAL, "tcgen05 must be 0 or 1");
  if (tcgen05 && P->L != 64)
    return fail(MUFFIN_EINVAL, "the tcgen05 spectral kernel needs 64 bands (plan has %d)", P->L);
  if (tcgen05 && P->p.precision != 0)
    return fail(MUFFIN_EINVAL, "the plan computes the spectral step in FP32");
  muffin::pi::drop_graphs_and_state(P);
  P->dct_tc = tcgen05;
  return MUFFIN_OK;
}

muffin_status muffin_plan_inject_timeout(muffin_plan P, int32_t on) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  muffin::pi::drop_graphs_and_state(P);
  P->inject_timeout = on ? 1 : 0;
  return MUFFIN_OK;
}

muffin_status muffin_plan_set_tuning(muffin_plan P, int32_t syn_packed, int32_t dct_ctas_per_sm) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  if (syn_packed < 0 || syn_packed > 3)
    return fail(MUFFIN_EINVAL, "syn_packed must be in 0..3 (got %d)", syn_packed);
  if (dct_ctas_per_sm < 0)
    return fail(MUFFIN_EINVAL, "dct_ctas_per_sm must be >= 0 (got %d)", dct_ctas_per_sm);
  muffin::pi::drop_graphs_and_state(P);
  P->syn_packed = syn_packed;
  P->dct_ctas = dct_ctas_per_sm;
  return MUFFIN_OK;
}

muffin_status muffin_plan_get_schedule(muffin_plan P, muffin_schedule *s) {
  if (!P || !s) return fail(MUFFIN_EINVAL, "NULL argument");
  s->syn_packed = P->syn_packed;
  s->dct_ctas_per_sm = P->dct_ctas;
  s->spectral_tcgen05 = P->dct_tc;
  s->grad_chunk = P->grad_chunk;
  s->fft_radix = P->fft_radix;
  s->group_order = P->group_order;
  s->ana_ring = P->ana_ring;
  s->ana_pipe = P->ana_pipe;
  return MUFFIN_OK;
}

muffin_status muffin_plan_set_schedule(muffin_plan P, const muffin_schedule *s) {
  if (!P || !s) return fail(MUFFIN_EINVAL, "NULL argument");
  if (s->syn_packed < 0 || s->syn_packed > 3 || s->dct_ctas_per_sm < 0 || s->grad_chunk < 0 ||
      (s->spectral_tcgen05 != 0 && s->spectral_tcgen05 != 1) ||
      (s->fft_radix != 16 && s->fft_radix != 8) || s->group_order < 0 || s->group_order > 2 ||
      s->ana_ring < 0 || s->ana_ring > 1 || s->ana_pipe < 0 || s->ana_pipe > 1)
    return fail(MUFFIN_EINVAL, "schedule value out of range");
  if (s->spectral_tcgen05 && P->L != 64)
    return fail(MUFFIN_EINVAL, "the tcgen05 spectral kernel needs 64 bands (plan has %d)", P->L);
  if (s->spectral_tcgen05 && P->p.precision != 0)
    return fail(MUFFIN_EINVAL, "the plan computes the spectral step in FP32");
  muffin::pi::drop_graphs_and_state(P);
  P->syn_packed = s->syn_packed;
  P->dct_ctas = s->dct_ctas_per_sm;
  P->dct_tc = s->spectral_tcgen05;
  P->grad_chunk = s->grad_chunk;
  P->fft_radix = P->n >= 64 ? s->fft_radix : 16;
  P->group_order = P->p.sure ? s->group_order : 0;
  P->ana_ring = s->ana_ring;
  P->ana_pipe = s->ana_pipe;
  return MUFFIN_OK;
}

muffin_status muffin_plan_autotune(muffin_plan P, const char *cache_path, muffin_tune_info *info) {
  if (!P) return fail(MUFFIN_EINVAL, "plan is NULL");
  const std::string key = shape_key(P);
  Choice c;
  bool cached = false;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) { c = it->second; cached = true; }
  }
  if (!cached && cache_path && file_lookup(cache_path, key, &c)) {
    cached = true;
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = c;
  }
  if (info) std::memset(info, 0, sizeof *info);
  if (cached) {
    muffin::pi::drop_graphs_and_state(P);
    apply(P, c);
    if (info) {
      info->syn_packed = c.syn_packed;
      info->dct_ctas_per_sm = c.dct_ctas;
      info->spectral_tcgen05 = P->dct_tc;
      info->grad_chunk = P->grad_chunk;
      info->fft_radix = P->fft_radix;
      info->group_order = P->group_order;
      info->ana_ring = P->ana_ring;
      info->ana_pipe = P->ana_pipe;
      info->from_cache = 1;
    }
    return MUFFIN_OK;
  }
  muffin::pi::drop_graphs_and_state(P);
  muffin_status s = tune(P, &c, info);
  muffin::pi::drop_graphs_and_state(P);
  if (s != MUFFIN_OK) return s;
  apply(P, c);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = c;
  }
  if (cache_path) file_append(cache_path, key, c);
  if (info) {
    info->syn_packed = c.syn_packed;
    info->dct_ctas_per_sm = c.dct_ctas;
    info->spectral_tcgen05 = P->dct_tc;
    info->grad_chunk = P->grad_chunk;
    info->fft_radix = P->fft_radix;
    info->group_order = P->group_order;
    info->ana_ring = P->ana_ring;
    info->ana_pipe = P->ana_pipe;
    info->from_cache = 0;
  }
  return MUFFIN_OK;
}

}  // extern "C"
