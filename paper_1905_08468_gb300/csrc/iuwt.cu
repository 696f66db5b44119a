// Isotropic undecimated wavelet transform (starlet), the alternative spatial
// dictionary W_s of Sec. 2.1, fused with the MUFFIN updates that consume it
// (Algorithm 2 and the derivative forms of Algorithms 3/4), like the
// Daubechies kernels in wavelet.cu:
//
//   analysis + dual update:  c_0 = 2x~ - x (chain mix of Algorithm 3),
//     c_{j+1} = S_j c_j, plane j gets w = c_j - c_{j+1}, plane J gets c_J;
//     p = u + sigma mu_l plane, u = sat(p) (eqs. stpp, stpu);
//   synthesis + primal prox: W^T u in Horner form
//     P_0 + S_0[(P_1 - P_0) + S_1[(P_2 - P_1) + ... + S_{J-1}(P_J - P_{J-1})]]
//     then m = x - tau (grad + mu_l s + t), x~ = (m)_+ (eqs. stpm, stpx).
//
// S_j is the separable B3 spline [1 4 6 4 1]/16 dilated by 2^j with periodic
// boundaries.  One launch per scale: a CTA loads its 16 x 32 tile of every
// chain with a 2 * 2^j halo (wrapped) into shared memory, smooths it along y
// then x, and does the scale's dual update (analysis) or Horner step
// (synthesis); the running image of the next scale goes to a ping-pong
// scratch.  The derivative chains use the primal's masks from the same
// thread (Pi(p) per coefficient, U(m) per pixel).  J <= 4 (halo <= 16).
#include <cuda_runtime.h>

#include <stdint.h>

#include "kernels.h"

namespace muffin {

namespace {

constexpr int IY = 16, IX = 32, INT = 256;   // output tile, threads
constexpr int IDMAX = 8;                       // largest dilation (J <= 4)
constexpr int IAY = IY + 4 * IDMAX, IAX = IX + 4 * IDMAX + 1;   // input tile (pitch odd)
constexpr int IBX = IX + 4 * IDMAX + 1;                          // vertical-pass pitch
// B3 spline tap m of [1 4 6 4 1] / 16
__device__ __forceinline__ constexpr float b3(int m) {
  return (m == 2 ? 6.f : (m == 1 || m == 3) ? 4.f : 1.f) * (1.f / 16.f);
}

constexpr size_t iuwt_smem(int ch) {
  return ((size_t)ch * IAY * IAX + (size_t)ch * IY * IBX) * sizeof(float);
}

struct IuwtArgs {
  int n, L, Lc, P, J, j;         // P = J + 1 planes per band, j = this scale
  int positivity;
  const float *xt, *x, *g, *t;   // iteration images [C][L][n][n]
  float *xt_out;                 // synthesis j = 0: x-tilde
  const float *in;               // operator input (analysis: x; synthesis: u)
  float *out;                    // synthesis operator output
  float *u;                      // [C][L][P][n][n] duals (analysis writes)
  const float *ur;               // duals read by the synthesis
  float *buf[2];                 // ping-pong running images [C][L][n][n]
  const float *beta;
  const DevScalars *sc;
};

__device__ __forceinline__ int wrap(int v, int n) { return v & (n - 1); }

// tile value of chain c at (yy, xx) for the source of scale j
template <int CH, int MODE>
__device__ __forceinline__ void ana_src(const IuwtArgs &a, int l, size_t pix, float mu,
                                        float (&w)[CH]) {
  const size_t NN = (size_t)a.n * a.n, CS = (size_t)a.L * NN;
  if (a.j == 0) {
    if (MODE == WAVE_TRANSFORM) {
      w[0] = a.in[(size_t)l * NN + pix];
    } else {
      float z[CH];
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const size_t i = c * CS + (size_t)l * NN + pix;
        z[c] = 2.f * a.xt[i] - a.x[i];
      }
      w[0] = z[0];
      if (CH == 3) { w[1] = fmaf(mu, z[1], z[0]); w[2] = z[2]; }
    }
  } else {
    const float *src = a.buf[a.j & 1];
#pragma unroll
    for (int c = 0; c < CH; ++c) w[c] = src[c * CS + (size_t)l * NN + pix];
  }
}

// separable B3 smoothing at dilation d of the resident tile A -> out[2] of
// the thread's two pixels (rows ry, ry + IY/2 of column rx)
template <int CH>
__device__ __forceinline__ void smooth_tile(const float *A, float *Bv, int d, int c,
                                            int ry, int rx, float (&out)[2]) {
  const float *Ac = A + c * IAY * IAX;
  float *Bc = Bv + c * IY * IBX;
  // vertical pass: IY rows x (IX + 4d) columns
  const int wcols = IX + 4 * d;
  for (int it = threadIdx.x; it < IY * wcols; it += INT) {
    const int r = it / wcols, col = it - r * wcols;
    float s = 0.f;
#pragma unroll
    for (int m = 0; m < 5; ++m) s = fmaf(b3(m), Ac[(r + m * d) * IAX + col], s);
    Bc[r * IBX + col] = s;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int r = ry + q * (IY / 2);
    float s = 0.f;
#pragma unroll
    for (int m = 0; m < 5; ++m) s = fmaf(b3(m), Bc[r * IBX + rx + m * d], s);
    out[q] = s;
  }
}

template <int CH, int MODE>
__global__ void __launch_bounds__(INT) k_iuwt_ana(IuwtArgs a) {
  extern __shared__ float ism[];
  float *A = ism;                       // [CH][IAY][IAX]
  float *Bv = A + CH * IAY * IAX;       // [CH][IY][IBX]
  const int n = a.n, d = 1 << a.j;
  const int ntx = (n + IX - 1) / IX;
  const int x0 = (blockIdx.x % ntx) * IX, y0 = (blockIdx.x / ntx) * IY;
  const int l = blockIdx.y;
  const size_t NN = (size_t)n * n, CS = (size_t)a.L * NN;
  float mu = 0.f, sbl = 1.f;
  if (MODE == WAVE_ITERATE) {
    const DevScalars &S = a.sc[l / a.Lc];
    mu = (float)S.mu;
    sbl = (float)(S.sigma * (double)a.beta[l]);
  }
  const int ay = IY + 4 * d, ax = IX + 4 * d;
  for (int it = threadIdx.x; it < ay * ax; it += INT) {
    const int r = it / ax, col = it - r * ax;
    const size_t pix = (size_t)wrap(y0 - 2 * d + r, n) * n + wrap(x0 - 2 * d + col, n);
    float w[CH];
    ana_src<CH, MODE>(a, l, pix, mu, w);
#pragma unroll
    for (int c = 0; c < CH; ++c) A[(c * IAY + r) * IAX + col] = w[c];
  }
  __syncthreads();
  const int rx = threadIdx.x % IX, ry = threadIdx.x / IX;   // rows ry, ry + 8
  const bool last = a.j == a.J - 1;
  uint32_t keep = 0;
#pragma unroll 1
  for (int c = 0; c < CH; ++c) {
    float cn[2];
    smooth_tile<CH>(A, Bv, d, c, ry, rx, cn);
    const float q = MODE == WAVE_ITERATE ? (c == 1 ? sbl : sbl * mu) : 1.f;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int r = ry + k * (IY / 2);
      const int yy = y0 + r, xx = x0 + rx;
      if (yy >= n || xx >= n) continue;
      const float cj = A[(c * IAY + r + 2 * d) * IAX + rx + 2 * d];
      const size_t pix = (size_t)yy * n + xx;
      float *up = a.u + ((size_t)(c * a.L + l) * a.P) * NN + pix;
      // planes j (detail) and, at the last scale, J (coarse)
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (s == 1 && !last) break;
        const float val = s == 0 ? cj - cn[k] : cn[k];
        float *uq = up + (size_t)(s == 0 ? a.j : a.J) * NN;
        if (MODE == WAVE_TRANSFORM) {
          *uq = val;
        } else {
          const float p = fmaf(q, val, *uq);
          const uint32_t bit = 1u << (2 * s + k);
          if (c == 0) {
            *uq = satf(p);
            if (fabsf(p) <= 1.0f) keep |= bit;
          } else {
            *uq = (keep & bit) ? p : 0.f;
          }
        }
      }
      if (!last) a.buf[(a.j + 1) & 1][c * CS + (size_t)l * NN + pix] = cn[k];
    }
    __syncthreads();
  }
}

// synthesis source of scale j: P_J - P_{J-1} at the coarsest step, else the
// running image of scale j + 1
template <int CH, int MODE>
__device__ __forceinline__ float syn_src(const IuwtArgs &a, int c, int l, size_t pix) {
  const size_t NN = (size_t)a.n * a.n, CS = (size_t)a.L * NN;
  if (a.j == a.J - 1) {
    const float *u = (MODE == WAVE_TRANSFORM ? a.in : a.ur) +
                     ((size_t)(c * a.L + l) * a.P) * NN + pix;
    return u[(size_t)a.J * NN] - u[(size_t)(a.J - 1) * NN];
  }
  return a.buf[(a.j + 1) & 1][c * CS + (size_t)l * NN + pix];
}

template <int CH, int MODE>
__global__ void __launch_bounds__(INT) k_iuwt_syn(IuwtArgs a) {
  extern __shared__ float ism[];
  float *A = ism;
  float *Bv = A + CH * IAY * IAX;
  const int n = a.n, d = 1 << a.j;
  const int ntx = (n + IX - 1) / IX;
  const int x0 = (blockIdx.x % ntx) * IX, y0 = (blockIdx.x / ntx) * IY;
  const int l = blockIdx.y;
  const size_t NN = (size_t)n * n, CS = (size_t)a.L * NN;
  const int ay = IY + 4 * d, ax = IX + 4 * d;
  for (int it = threadIdx.x; it < ay * ax; it += INT) {
    const int r = it / ax, col = it - r * ax;
    const size_t pix = (size_t)wrap(y0 - 2 * d + r, n) * n + wrap(x0 - 2 * d + col, n);
#pragma unroll
    for (int c = 0; c < CH; ++c) A[(c * IAY + r) * IAX + col] = syn_src<CH, MODE>(a, c, l, pix);
  }
  __syncthreads();
  const int rx = threadIdx.x % IX, ry = threadIdx.x / IX;
  float o[CH][2];
#pragma unroll 1
  for (int c = 0; c < CH; ++c) {
    float sr[2];
    smooth_tile<CH>(A, Bv, d, c, ry, rx, sr);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int yy = y0 + ry + k * (IY / 2), xx = x0 + rx;
      o[c][k] = 0.f;
      if (yy >= n || xx >= n) continue;
      const size_t pix = (size_t)yy * n + xx;
      const float *u = (MODE == WAVE_TRANSFORM ? a.in : a.ur) +
                       ((size_t)(c * a.L + l) * a.P) * NN + pix;
      if (a.j > 0) {
        const float v = sr[k] + u[(size_t)a.j * NN] - u[(size_t)(a.j - 1) * NN];
        a.buf[a.j & 1][c * CS + (size_t)l * NN + pix] = v;
      } else {
        o[c][k] = u[0] + sr[k];
      }
    }
    __syncthreads();
  }
  if (a.j > 0) return;
  const float mu = (MODE == WAVE_ITERATE) ? (float)a.sc[l / a.Lc].mu : 0.f;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int yy = y0 + ry + k * (IY / 2), xx = x0 + rx;
    if (yy >= n || xx >= n) continue;
    const size_t i0 = (size_t)l * NN + (size_t)yy * n + xx;
    if (MODE == WAVE_TRANSFORM) {
      a.out[i0] = o[0][k];
      continue;
    }
    // W^T of chain 1 by linearity: W^T u + mu W^T u'_mu (Algorithm 3)
    float acc[CH];
    acc[0] = o[0][k];
    if (CH == 3) { acc[1] = fmaf(mu, o[1][k], o[0][k]); acc[2] = o[2][k]; }
    const float tau = (float)a.sc[l / a.Lc].tau;
    const float bl = a.beta[l];
    bool keep = true;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const float sc = (CH == 3 && c == 1) ? bl : bl * mu;   // mu_l, beta_l, mu_l
      const size_t i = c * CS + i0;
      const float m = a.x[i] - tau * (a.g[i] + sc * acc[c] + a.t[i]);
      if (c == 0) keep = !a.positivity || m > 0.f;
      a.xt_out[i] = keep ? m : 0.f;
    }
  }
}

inline int itiles(int n) { return ((n + IX - 1) / IX) * ((n + IY - 1) / IY); }

template <typename K>
void set_smem(K kern, size_t bytes) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int CH, int MODE>
cudaError_t ana_all(const WaveArgs &w, IuwtArgs a, cudaStream_t st) {
  static bool attr = false;
  if (!attr) { set_smem(k_iuwt_ana<CH, MODE>, iuwt_smem(CH)); attr = true; }
  const double vox = (double)CH * w.L * w.n * w.n;
  for (int j = 0; j < w.J; ++j) {
    a.j = j;
    const double bytes = vox * ((j == 0 && MODE == WAVE_ITERATE ? 8.0 : 4.0) +
                                (MODE == WAVE_ITERATE ? 8.0 : 4.0) * (j == w.J - 1 ? 2 : 1) +
                                (j == w.J - 1 ? 0.0 : 4.0));
    ProfScope ps(w.prof, "iuwt_ana_dual", bytes, vox * 22.0, st);
    k_iuwt_ana<CH, MODE><<<dim3(itiles(w.n), w.L), INT, iuwt_smem(CH), st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int CH, int MODE>
cudaError_t syn_all(const WaveArgs &w, IuwtArgs a, cudaStream_t st) {
  static bool attr = false;
  if (!attr) { set_smem(k_iuwt_syn<CH, MODE>, iuwt_smem(CH)); attr = true; }
  const double vox = (double)CH * w.L * w.n * w.n;
  for (int j = w.J - 1; j >= 0; --j) {
    a.j = j;
    const double bytes = vox * ((j == w.J - 1 ? 8.0 : 4.0) + 8.0 * (j > 0) + 4.0 * (j == 0) +
                                (j > 0 ? 4.0 : (MODE == WAVE_ITERATE ? 16.0 : 4.0)));
    ProfScope ps(w.prof, j == 0 ? "iuwt_syn_prox" : "iuwt_syn", bytes, vox * 22.0, st);
    k_iuwt_syn<CH, MODE><<<dim3(itiles(w.n), w.L), INT, iuwt_smem(CH), st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

IuwtArgs base_args(const WaveArgs &w, int C) {
  IuwtArgs a{};
  a.n = w.n; a.L = w.L; a.Lc = w.Lc > 0 ? w.Lc : w.L; a.P = w.J + 1; a.J = w.J;
  a.beta = w.beta; a.sc = w.sc;
  const size_t cl = (size_t)C * w.L * w.n * w.n;
  a.buf[0] = w.scratch;
  a.buf[1] = w.scratch + cl;
  return a;
}

}  // namespace

cudaError_t iuwt_analysis_dual(const WaveArgs &w, const Group &gr, cudaStream_t st) {
  IuwtArgs a = base_args(w, gr.C);
  a.xt = gr.xt; a.x = gr.x; a.u = gr.u;
  if (gr.C == 3) return ana_all<3, WAVE_ITERATE>(w, a, st);
  return ana_all<1, WAVE_ITERATE>(w, a, st);
}

cudaError_t iuwt_synthesis_prox(const WaveArgs &w, const Group &gr, int positivity,
                                cudaStream_t st) {
  IuwtArgs a = base_args(w, gr.C);
  a.x = gr.x; a.g = gr.g; a.t = gr.t; a.ur = gr.u; a.xt_out = gr.xt;
  a.positivity = positivity;
  if (gr.C == 3) return syn_all<3, WAVE_ITERATE>(w, a, st);
  return syn_all<1, WAVE_ITERATE>(w, a, st);
}

cudaError_t iuwt_analysis_op(const WaveArgs &w, const float *x, float *u, cudaStream_t st) {
  IuwtArgs a = base_args(w, 1);
  a.in = x; a.u = u;
  return ana_all<1, WAVE_TRANSFORM>(w, a, st);
}

cudaError_t iuwt_synthesis_op(const WaveArgs &w, const float *u, float *x, cudaStream_t st) {
  IuwtArgs a = base_args(w, 1);
  a.in = u; a.out = x;
  return syn_all<1, WAVE_TRANSFORM>(w, a, st);
}

}  // namespace muffin
