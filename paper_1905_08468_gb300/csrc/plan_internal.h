// Plan object shared by the C ABI (plan.cu) and the request server (serve.cu).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/muffin.h"
#include "kernels.h"

namespace muffin {

muffin_status fail(muffin_status s, const char *fmt, ...);

#define MUFFIN_CK(expr)                                                          \
  do {                                                                           \
    cudaError_t e_ = (expr);                                                     \
    if (e_ != cudaSuccess)                                                       \
      return ::muffin::fail(                                                     \
          e_ == cudaErrorMemoryAllocation ? MUFFIN_ENOMEM : MUFFIN_ECUDA,        \
          "%s: %s", #expr, cudaGetErrorString(e_));                              \
  } while (0)

bool is_device_ptr(const void *p);

}  // namespace muffin

// A plan holds B cubes ("slots") of L bands of n x n pixels, stored one
// after the other along the band axis (Lt = B L bands in all), so every
// spatial kernel runs over all of them in one launch and the spectral
// kernel runs one pixel tile of one cube per CTA.
struct muffin_plan_s {
  muffin_params p{};
  int n = 0, L = 0, K = 0, J = 0, Lp = 0, Cmax = 1, B = 1, Lt = 0;
  int dict = 0;        // 0: Daubechies union (K bases), 1: IUWT (K = J + 1 planes)
  double wsn2 = 0;     // ||W_s||^2 of the step condition
  size_t N = 0;      // pixels per band
  size_t NLc = 0;    // voxels per cube
  size_t NL = 0;     // voxels of all cubes
  cudaStream_t st = nullptr;   // caller's stream
  cudaStream_t ws = nullptr;   // plan's own work stream (graph capture)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaStream_t ws2 = nullptr;                          // second work stream (ADA-PT)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;    // its fork and join
  std::vector<void *> allocs;
  size_t bytes = 0;

  double2 *hhat = nullptr, *w64a = nullptr, *w64b = nullptr;
  float *kspec = nullptr;
  float2 *tw32 = nullptr;
  double2 *tw64 = nullptr;
  float *chi = nullptr, *clo = nullptr, *cthi = nullptr, *ctlo = nullptr;
  float2 *ftab = nullptr;   // FP32 spectral step tables (precision 1)
  int ftw_len = 0;
  float *alpha = nullptr, *beta = nullptr;
  muffin::DevScalars *sc = nullptr;   // [B]
  double *cube_const = nullptr;       // [B][4] for the theta update
  int *rec_count = nullptr;           // device counter of trace records
  double *dred = nullptr;             // reduction scratch
  double *wband = nullptr;            // [Lt]
  double *records = nullptr;          // [max_records][B][7]
  int max_records = 0;
  float2 *S = nullptr;
  float *llscr = nullptr;
  float2 *S2 = nullptr;        // scratch of the group on the second stream
  float *llscr2 = nullptr;
  size_t lvl_off[16] = {};
  muffin::Group grp[2];
  float *grp_x0[2] = {nullptr, nullptr};   // x buffer at allocation (graph parity)
  float *b = nullptr, *bbar = nullptr, *htd = nullptr;
  float *stage_a = nullptr, *stage_b = nullptr;
  float *op_in = nullptr, *op_out = nullptr, *op_b = nullptr;
  double *mon = nullptr;              // monitor reduction scratch and outputs
  float *ydev = nullptr;              // dirty cube kept for the monitor's objective
  bool have_y = false;
  std::vector<float> beta_h;          // band weights (host copy)
  muffin_monitor_params mon_p{};      // convergence monitor settings
  std::vector<muffin_monitor_record> mon_rec;   // records of the last call

  muffin::Prof prof;
  bool profiling = false;
  bool use_graphs = true;
  int syn_packed = 0;     // synthesis variant bits (see WaveArgs::syn_packed)
  int ana_ring = 0;       // analysis U staging (see WaveArgs::ana_ring)
  int ana_pipe = 0;       // level-1 analysis kernel (see WaveArgs::ana_pipe)
  int dct_ctas = 0;       // spectral kernel CTAs per SM (0: all resident)
  int dct_tc = 0;         // spectral step on tcgen05 (L = 64)
  int grad_chunk = 0;     // images per pass of the gradient FFTs (0: all at once)
  int fft_radix = 16;     // largest radix of the gradient FFT plan (16, or 8 from n = 64)
  int group_order = 0;    // ADA-PT: 0 group after group, 1 phase by phase, 2 concurrent streams
  int tw_len16 = 0;       // entries of the radix-16 twiddle tables (the radix-8 ones follow)
  int inject_timeout = 0; // test hook (muffin_plan_inject_timeout)
  int *kerr = nullptr;    // device flag: a bounded tensor-core wait gave up
  // (parity, runs of cubes) -> two plain iterations
  std::map<std::pair<int, std::vector<std::pair<int, int>>>, cudaGraphExec_t> gplain;
  cudaGraphExec_t gsure[2] = {nullptr, nullptr};
  int gsure_window = 0, gsure_reset = -1;
  double gsure_eta[2] = {0, 0}, gsure_tmin = 0;

  std::vector<double> lips, Asum, Amax2, Bsum, Bmax2, psc, mu, gamma;
  bool have_b = false, have_state = false, have_sure_state = false;
  bool vis_b = false;     // b and the spectra come from loaded visibilities
  long long k_done = 0;

  muffin::Prof *pp() { return profiling ? &prof : nullptr; }
  // twiddle tables of the selected FFT plan
  const float2 *tw() const { return fft_radix == 8 && n >= 64 ? tw32 + tw_len16 : tw32; }

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

  ~muffin_plan_s();

  double lnorm2(int c, double m, double g) const {
    if (p.step_rule == 0) return wsn2 * m * m * Bsum[c] + g * g * Asum[c];
    return wsn2 * m * m * Bmax2[c] + g * g * Amax2[c];
  }
  double tau_for(int c, double m, double g) const {
    if (p.tau > 0) return p.tau;
    return p.tau_safety / (0.5 * lips[c] + p.sigma * lnorm2(c, m, g));
  }
  muffin::WaveArgs wave(int C) {
    muffin::WaveArgs w{};
    w.n = n; w.L = Lt; w.Lc = L; w.K = K; w.J = J; w.C = C; w.dict = dict;
    w.beta = beta; w.sc = sc; w.scratch = llscr;
    for (int j = 0; j < 16; ++j) w.lvl_off[j] = lvl_off[j];
    w.syn_packed = syn_packed;
    w.ana_ring = ana_ring;
    w.ana_pipe = ana_pipe;
    w.prof = pp();
    return w;
  }
  muffin::DctArgs dct(int C) {
    muffin::DctArgs d{};
    d.n = n; d.L = L; d.Lp = Lp; d.C = C; d.B = B;
    d.chi = chi; d.clo = clo; d.cthi = cthi; d.ctlo = ctlo;
    d.alpha = alpha; d.sc = sc;
    d.ctas_per_sm = dct_ctas;
    d.tc = dct_tc; d.err = kerr; d.inject_timeout = inject_timeout;
    d.f32 = p.precision == 1; d.ftab = ftab; d.ftw_len = ftw_len;
    d.prof = pp();
    return d;
  }
};

namespace muffin {
namespace pi {

// device bytes a plan with parameters p allocates (p valid)
size_t estimate_bytes(const muffin_params *p);
// creation; psf may be NULL (slots loaded later with load_psf)
muffin_status create(const muffin_params *p, const float *psf, const float *alpha,
                     const float *beta, void *stream, muffin_plan *out);
// PSF spectra, |h_hat|^2 / n^2 and beta of cubes [b0, b1); psf holds b1-b0 cubes
muffin_status load_psf(muffin_plan P, int b0, int b1, const float *psf);
// b = H^T y for cubes [b0, b1) (FP64); dirty holds b1-b0 cubes
muffin_status load_dirty(muffin_plan P, int b0, int b1, const float *dirty);
// group g: cubes [b0, b1) restart from X0 (device, b1-b0 cubes; NULL = 0), U = V = T = 0
muffin_status reset_cubes(muffin_plan P, int g, int b0, int b1, const float *x0_dev);
// (mu, gamma) of cubes [b0, b1) and their tau (host arrays of b1-b0 values)
muffin_status set_theta(muffin_plan P, int b0, int b1, const double *mu, const double *gamma);
// `iters` plain iterations of group 0 on the runs [c0, c1) of cubes (all
// cubes when runs is empty), on the work stream
muffin_status run_plain(muffin_plan P, int iters, const std::vector<std::pair<int, int>> &runs);
// copy X of cubes [b0, b1) of group 0 to dst (host or device)
muffin_status fetch_x(muffin_plan P, int b0, int b1, float *dst);
// order the work stream after the caller's stream / the caller's after it
muffin_status enter(muffin_plan P);
muffin_status leave(muffin_plan P, bool sync);
// one iteration of every chain group the plan advances (work stream, direct
// launches); used by the tuner
muffin_status iterate_all(muffin_plan P);
// destroy the captured graphs (they bake in kernel variants) and forget the
// iterate state, so the next solve starts cold
void drop_graphs_and_state(muffin_plan P);

}  // namespace pi
}  // namespace muffin
