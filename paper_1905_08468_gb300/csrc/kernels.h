// Host-side launchers of the MUFFIN kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace muffin {

// Per-kernel timing with CUDA events on the launching stream.  Launchers
// call begin()/end() around every kernel when a profiler is attached; the
// plan resolves the event pairs at the end of each API call.
struct Prof {
  struct Stat {
    std::string name;
    long long launches = 0;
    double total_ms = 0, bytes = 0, flops = 0;   // bytes/flops per launch
  };
  struct Pending { int id; cudaEvent_t a, b; };
  std::vector<Stat> stats;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;

  int find(const char *name, double bytes, double flops) {
    for (size_t i = 0; i < stats.size(); ++i)
      if (stats[i].name == name && stats[i].bytes == bytes) return (int)i;
    Stat s;
    s.name = name; s.bytes = bytes; s.flops = flops;
    stats.push_back(s);
    return (int)stats.size() - 1;
  }
  cudaEvent_t take() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  // a bracket returns its (stat, start event) token, so brackets may nest
  // (an aggregate around several launches, e.g. the chunks of the gradient)
  Pending begin(const char *name, double bytes, double flops, cudaStream_t st) {
    if (pending.size() >= 2048) resolve();
    Pending t{find(name, bytes, flops), take(), nullptr};
    cudaEventRecord(t.a, st);
    return t;
  }
  void end(Pending t, cudaStream_t st) {
    t.b = take();
    cudaEventRecord(t.b, st);
    pending.push_back(t);
  }
  void resolve() {
    if (pending.empty()) return;
    cudaEventSynchronize(pending.back().b);
    for (const Pending &p : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        stats[p.id].total_ms += ms;
        stats[p.id].launches += 1;
      }
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
    cudaGetLastError();
  }
  void reset() { resolve(); stats.clear(); }
  ~Prof() {
    resolve();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

// RAII bracket used by the launchers
struct ProfScope {
  Prof *p;
  cudaStream_t st;
  Prof::Pending t{};
  ProfScope(Prof *p_, const char *name, double bytes, double flops, cudaStream_t s)
      : p(p_), st(s) { if (p) t = p->begin(name, bytes, flops, st); }
  ~ProfScope() { if (p) p->end(t, st); }
};

// Records msg as the thread's muffin_last_error() text and returns s (plan.cu).
int set_last_error_code(int s, const char *msg);

// ------------------------------------------------------------ FFT (fft_conv.cu)
// FP32 gradient pipeline: g[c][l] = H_l^T H_l x[c][l] - (c == 0 && b ? b[l] : 0)
// for nimg = C*L images.  S: spectrum scratch [nimg][n/2+1][n] float2.
// kspec: [L][n/2+1][n] = |h_hat_l(ky, kx)|^2 / n^2 (kx-major).
// chunk > 0: the three passes run over `chunk` images at a time (S then
// needs room for chunk images only and stays in L2 between the passes);
// chunk <= 0: each pass over all images at once.
// radix 16 (default) or 8 (n >= 64): the largest radix of the FFT plan; tw
// must hold that plan's twiddle tables (fft32_tables with the same radix).
cudaError_t launch_gradient(const float *x, float *g, const float *b,
                            float2 *S, const float *kspec, const float2 *tw,
                            int n, int L, int C, cudaStream_t st,
                            Prof *prof = nullptr, int chunk = 0, int radix = 16);

// Stage twiddle tables of the FP32 gradient FFT for side n (host side), for
// the plan whose largest radix is `radix`.
int fft32_table_len(int n, int radix = 16);
void fft32_tables(int n, float2 *tab, int radix = 16);

// FP64 helpers used when a plan or a call is set up.
// In-place 2D DFT of nimg complex n x n images; inverse is unnormalised.
cudaError_t fft2d_c64(double2 *data, double2 *tmp, int n, int nimg, bool inverse,
                      const double2 *tw64, cudaStream_t st);
cudaError_t real_to_c64(const float *in, double2 *out, size_t count,
                        cudaStream_t st);
// a *= conj(h) elementwise (count elements)
cudaError_t mul_conj_c64(double2 *a, const double2 *h, size_t count,
                         cudaStream_t st);
// out = (float)(scale * in.x)
cudaError_t c64_real_to_f32(const double2 *in, float *out, double scale,
                            size_t count, cudaStream_t st);
// kspec[l][kx][ky] = |hh[l][ky][kx]|^2 * scale for kx < n/2+1
cudaError_t make_kspec(const double2 *hh, float *kspec, double scale, int n,
                       int L, cudaStream_t st);

// ------------------------------------------------------------ reductions (reduce.cu)
// out[0] = max |hh|^2 over count complex values (FP64); scratch >= 1024 doubles
cudaError_t max_abs2_c64(const double2 *hh, size_t count, double *scratch,
                         double *out, cudaStream_t st);
// per-band sum of squares: out[l] = sum y[l]^2 (FP64)
cudaError_t band_sumsq(const float *y, int L, size_t per_band, double *out,
                       cudaStream_t st);
// alpha[b][n] = 1 / (||x[b][:, n]||_2 + eps) over the L bands of cube b (FP64 sum)
cudaError_t pixel_weights(const float *x, int B, int L, size_t N, double eps, float *alpha,
                          cudaStream_t st);
// ybar = y + eps * delta ; hd unchanged
cudaError_t axpy_f32(const float *y, const float *d, float eps, float *out,
                     size_t count, cudaStream_t st);

// SURE statistics at a window end (Eqs. SUGAR, PSURE0, rewritten with H^T):
//   s0 = <grad, x'_mu>        s1 = <grad, x'_gamma>
//   s2 = sum_l w_l <xbar'_mu - x'_mu, H^T delta>
//   s3 = sum_l w_l <xbar'_gamma - x'_gamma, H^T delta>
//   s4 = <x, grad - b>         s5 = sum_l w_l <xbar - x, H^T delta>
// with w_l = 2 sigma_l^2 / eps.  ga/gb are the y- and ybar-groups (C = 3),
// grad the gradient at the current x of the y-group primal.
// partials: [nblocks][6] doubles, deterministic two-pass reduction.
struct SureStatsArgs {
  const float *grad;  // [L][n][n] gradient at the y-group primal
  const float *x;     // y-group X [3][L][n][n] (primal, d/dmu, d/dgamma)
  const float *xb;    // ybar-group X [3][L][n][n]
  const float *b;     // [L][n][n] H^T y
  const float *htd;   // [L][n][n] H^T delta
  const double *wband;  // [L] 2 sigma_l^2 / eps
  int n, L;
};
// nblocks = blocks per band (partials are band-major)
cudaError_t sure_stats(const SureStatsArgs &a, double *partials, int *nblocks,
                       cudaStream_t st);

// Theta update (Eq. adaptgrad) run on the device, one block per cube, then
// the record counter is advanced (so the same launches can be replayed).
struct ThetaUpdateArgs {
  int B;                   // cubes
  DevScalars *sc;          // [B] in/out
  const double *partials;  // [B][nb_per_cube][6] (bands of a cube are contiguous)
  int nb_per_cube;
  double *record;          // out: cube b of record r at record + (r*B + b)*7:
  int *rec_count;          //   {0, mu, gamma, sugar_mu, sugar_gamma, psure, tau}
                           //   (theta before the update); r = *rec_count
  double eta_mu, eta_gamma, theta_min;
  // per cube: {sum_l ||y_l||^2 - N sum_l sigma_l^2, beta, Bsum, Asum} with
  // tau = safety / (beta/2 + sigma * (K * mu^2 * Bsum + gamma^2 * Asum))
  const double *cube_const;
  double safety, K;
  double tau_fixed;        // > 0: tau stays at this value (the plan's override)
};
cudaError_t theta_update(const ThetaUpdateArgs &a, cudaStream_t st);

// ------------------------------------------------------------ monitor (monitor.cu)
// Doubles of scratch the monitor reductions need for L bands: partials
// [L][16][3], then the outputs state [L][3], residual [L], |W_s x| [L],
// alpha |W_lambda x| [L], input scan [L][3], noise estimate [L][3].
size_t monitor_scratch_doubles(int L);
// out[l][0..2] = {sum (x - xo)^2, sum xo^2 (sum x^2 when xo is NULL), number
// of NaN/Inf entries of x} over the N values of band l (FP64)
cudaError_t mon_state(const float *x, const float *xo, int L, size_t N, double *scratch,
                      double *out, cudaStream_t st);
// out[l] = sum_i (scale * w[l][i].x - y[l][i])^2 (FP64)
cudaError_t mon_resid2(const double2 *w, const float *y, double scale, int L, size_t N,
                       double *scratch, double *out, cudaStream_t st);
// out[l] = sum_i a_i |u[l][i]| over per_band values, a_i = alpha[(l / Lc) N + i mod N]
// (or 1 when alpha is NULL)
cudaError_t mon_abs(const float *u, int L, size_t per_band, const float *alpha, int Lc,
                    size_t N, double *scratch, double *out, cudaStream_t st);
// a *= h elementwise (complex FP64)
cudaError_t mul_c64(double2 *a, const double2 *h, size_t count, cudaStream_t st);
// z = 2 xt - x (the spectral step's input, Alg. 2 eq. vt)
cudaError_t twice_minus(const float *xt, const float *x, float *z, size_t count,
                        cudaStream_t st);

// ------------------------------------------------------------ noise (noise.cu)
// MAD noise level of L images y [L][n][n]: var[l] = (MAD / Phi^-1(3/4))^2 of
// the finest Haar high-high band; d_scratch holds L (n/2)^2 floats, med and
// mad L doubles each
cudaError_t noise_mad(const float *y, int n, int L, float *d_scratch, double *med,
                      double *mad, double *var, cudaStream_t st);

// ------------------------------------------------------------ wavelets (wavelet.cu)
// Filters db1..db8: h, g taps (g[i] = (-1)^i h[2p-1-i]) uploaded to constant memory.
cudaError_t upload_filters(const double h[8][16]);

enum WaveMode { WAVE_TRANSFORM = 0, WAVE_ITERATE = 1 };

struct WaveArgs {
  int n, L, K, J, C;       // L = all bands of all cubes of the batch
  int Lc;                  // bands per cube (0: one cube of L bands)
  const float *beta;       // [L] band weights
  const DevScalars *sc;    // [L / Lc] per cube: mu, gamma, tau, sigma
  float *scratch;          // LL scratch: level j (1 <= j < J) holds
                           // [C][L][K][n>>j][n>>j] at scratch + lvl_off[j]
  size_t lvl_off[16];
  int dict;                // 0: union of K Daubechies bases, 1: IUWT (K = J + 1 planes)
  int ana_ring;            // analysis of the size-specialised levels: 1 stages the
                           // U detail tiles in a shared-memory ring by cp.async
  int ana_pipe;            // level-1 analysis (iteration, J > 1): 1 runs the
                           // chain-major kernel with one barrier per step
  int syn_packed;          // synthesis variant: bit 0 coarse levels, bit 1
                           // level 1 (0 scalar row pass, 1 packed row pairs)
  Prof *prof;              // optional per-kernel timing
};

// Synthesis + primal prox (Alg. 2 eqs. adjointspat2, stpm, stpx and the
// derivative forms of Algs. 3/4): reads gr.u, gr.x, gr.g, gr.t -> gr.xt.
cudaError_t wavelet_synthesis_prox(const WaveArgs &w, const Group &gr,
                                   int positivity, cudaStream_t st);
// Analysis + spatial dual update (eqs. stpp, stpu and derivative forms):
// reads gr.xt, gr.x, gr.u -> gr.u.
cudaError_t wavelet_analysis_dual(const WaveArgs &w, const Group &gr,
                                  cudaStream_t st);
// IUWT (starlet) forms of the four calls above and below (iuwt.cu); the
// scratch holds two [C][L][n][n] running images.  J >= 1.
cudaError_t iuwt_analysis_dual(const WaveArgs &w, const Group &gr, cudaStream_t st);
cudaError_t iuwt_synthesis_prox(const WaveArgs &w, const Group &gr, int positivity,
                                cudaStream_t st);
cudaError_t iuwt_analysis_op(const WaveArgs &w, const float *x, float *u, cudaStream_t st);
cudaError_t iuwt_synthesis_op(const WaveArgs &w, const float *u, float *x, cudaStream_t st);
// Operators: u = W_s x ; x = W_s^T u (C = 1, no weights).
cudaError_t wavelet_analysis_op(const WaveArgs &w, const float *x, float *u,
                                cudaStream_t st);
cudaError_t wavelet_synthesis_op(const WaveArgs &w, const float *u, float *x,
                                 cudaStream_t st);

// ------------------------------------------------------------ DCT (dct.cu)
struct DctArgs {
  int n, L, Lp, C;         // L = bands per cube, Lp = L rounded up to 16
  size_t npix;             // pixels per band: 0 = n * n; else a block of pixels
  int B;                   // cubes in the batch (band-major, cube after cube)
  const float *chi, *clo;  // [Lp][Lp] C split in TF32 hi + lo (zero padded)
  const float *cthi, *ctlo;// [Lp][Lp] C^T split
  const float *alpha;      // [B][n*n] pixel weights
  const DevScalars *sc;    // [B]
  int ctas_per_sm;         // persistent spectral grid: CTAs per SM (0: max resident)
  int tc;                  // 1: tcgen05 kernel (L = 64), 0: mma.sync kernel
  int *err;                // device flag raised when a tensor-core wait gives up
  int inject_timeout;      // test hook: the tcgen05 kernel issues no products
  int f32;                 // 1: FP32 fast DCT on the CUDA cores (dct_f32.cu)
  const float2 *ftab;      // its tables: DFT stage twiddles, then (cos, sin)(pi k / 2L)
  int ftw_len;             // stage twiddle entries at the head of ftab
  Prof *prof;              // optional per-kernel timing
};
// Spectral dual update and back-projection (Alg. 2 eqs. vt, v, upt and the
// derivative forms of Algs. 3/4): reads gr.xt, gr.x, gr.v -> gr.v, gr.t.
cudaError_t dct_dual(const DctArgs &d, const Group &gr, cudaStream_t st);
// The same step on the tcgen05 tensor cores (dct_tc.cu), L = Lp = 64.
cudaError_t dct_dual_tc(const DctArgs &d, const Group &gr, int *err, cudaStream_t st);
// Operator: out^n = C in^n (inverse = 0) or C^T in^n (inverse = 1).
cudaError_t dct_op(const DctArgs &d, const float *in, float *out, int inverse,
                   cudaStream_t st);
// The FP32 forms (L a power of two in [2, 1024]) and their tables:
// dct_f32_table_len(L) float2 entries, filled by dct_f32_tables.
cudaError_t dct_dual_f32(const DctArgs &d, const Group &gr, cudaStream_t st);
cudaError_t dct_op_f32(const DctArgs &d, const float *in, float *out, int inverse,
                       cudaStream_t st);
int dct_f32_table_len(int L);
void dct_f32_tables(int L, float2 *tab);

// ------------------------------------------------------------ visibilities (visibility.cu)
// h_hat = sqrt((m[k] + m[-k]) / 2) of nimg weight images; chk = m with NaN
// where m < 0
cudaError_t vis_weights(const float *m, double2 *hh, float *chk, int n, int nimg,
                        cudaStream_t st);
// count complex visibilities (re, im float pairs) -> FP64 complex
cudaError_t vis_to_c64(const float *vis, double2 *out, size_t count, cudaStream_t st);

}  // namespace muffin
