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
// boundaries.  One launch per scale, specialised on the dilation: a CTA
// loads its 32 x 64 tile of every chain with a 2 * 2^j halo (wrapped) into
// shared memory (four items per thread in flight), smooths it along y then
// x, and does the scale's dual update (analysis) or Horner step
// (synthesis); the running image of the next scale goes to a ping-pong
// scratch.  The derivative chains use the primal's masks from the same
// thread (Pi(p) per coefficient, U(m) per pixel).  J <= 4 (halo <= 16).
#include <cuda_runtime.h>

#include <stdint.h>

#include "kernels.h"

namespace muffin {

namespace {

constexpr int IY = 32, IX = 64, INT = 256;   // output tile, threads
constexpr int IQ = IY * IX / INT;              // outputs per thread (one column)

// B3 spline tap m of [1 4 6 4 1] / 16
__device__ __forceinline__ constexpr float b3(int m) {
  return (m == 2 ? 6.f : (m == 1 || m == 3) ? 4.f : 1.f) * (1.f / 16.f);
}

// shared-memory geometry of a dilation D: input tile [IY + 4D][PA], vertical
// pass [IY][PA] (odd pitch), per chain
template <int D> struct Geo {
  static constexpr int AY = IY + 4 * D, AX = IX + 4 * D;
  static constexpr int PITCH = (AX & 1) ? AX : AX + 1;
};
template <int D>
constexpr size_t iuwt_smem(int ch) {
  return (size_t)ch * (Geo<D>::AY + IY) * Geo<D>::PITCH * sizeof(float);
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

// tile value of chain c at pixel pix for the source of analysis scale j
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

// synthesis source of scale j: P_J - P_{J-1} at the coarsest step, else the
// running image of scale j + 1
template <int CH, int MODE>
__device__ __forceinline__ void syn_src(const IuwtArgs &a, int l, size_t pix, float (&w)[CH]) {
  const size_t NN = (size_t)a.n * a.n, CS = (size_t)a.L * NN;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    if (a.j == a.J - 1) {
      const float *u = (MODE == WAVE_TRANSFORM ? a.in : a.ur) +
                       ((size_t)(c * a.L + l) * a.P) * NN + pix;
      w[c] = u[(size_t)a.J * NN] - u[(size_t)(a.J - 1) * NN];
    } else {
      w[c] = a.buf[(a.j + 1) & 1][c * CS + (size_t)l * NN + pix];
    }
  }
}

// fill the wrapped input tile of every chain; LB items per thread per round
// so their loads are in flight together
template <int CH, int D, bool ANA, int MODE>
__device__ __forceinline__ void load_tile(const IuwtArgs &a, float *A, int y0, int x0, int l,
                                          float mu) {
  using G = Geo<D>;
  constexpr int LB = 4;
  const int n = a.n;
  constexpr int items = G::AY * G::AX;
  for (int base = threadIdx.x; base < items; base += LB * INT) {
    float w[LB][CH];
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int it = base + q * INT;
      if (it < items) {
        const int r = it / G::AX, col = it - r * G::AX;
        const size_t pix = (size_t)wrap(y0 - 2 * D + r, n) * n + wrap(x0 - 2 * D + col, n);
        if (ANA) ana_src<CH, MODE>(a, l, pix, mu, w[q]);
        else syn_src<CH, MODE>(a, l, pix, w[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int it = base + q * INT;
      if (it < items) {
        const int r = it / G::AX, col = it - r * G::AX;
#pragma unroll
        for (int c = 0; c < CH; ++c) A[(c * G::AY + r) * G::PITCH + col] = w[q][c];
      }
    }
  }
}

// separable B3 smoothing at dilation D of chain c's resident tile -> out[q]
// at the thread's pixels (rows ry + q * INT / IX of column rx)
template <int D>
__device__ __forceinline__ void smooth_tile(const float *A, float *Bv, int c, int ry, int rx,
                                            float (&out)[IQ]) {
  using G = Geo<D>;
  const float *Ac = A + c * G::AY * G::PITCH;
  float *Bc = Bv + c * IY * G::PITCH;
  for (int it = threadIdx.x; it < IY * G::AX; it += INT) {
    const int r = it / G::AX, col = it - r * G::AX;
    float s = 0.f;
#pragma unroll
    for (int m = 0; m < 5; ++m) s = fmaf(b3(m), Ac[(r + m * D) * G::PITCH + col], s);
    Bc[r * G::PITCH + col] = s;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < IQ; ++q) {
    const int r = ry + q * (INT / IX);
    float s = 0.f;
#pragma unroll
    for (int m = 0; m < 5; ++m) s = fmaf(b3(m), Bc[r * G::PITCH + rx + m * D], s);
    out[q] = s;
  }
}

template <int CH, int MODE, int D>
__global__ void __launch_bounds__(INT) k_iuwt_ana(IuwtArgs a) {
  using G = Geo<D>;
  extern __shared__ float ism[];
  float *A = ism;                        // [CH][AY][PITCH]
  float *Bv = A + CH * G::AY * G::PITCH; // [CH][IY][PITCH]
  const int n = a.n;
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
  load_tile<CH, D, true, MODE>(a, A, y0, x0, l, mu);
  __syncthreads();
  const int rx = threadIdx.x % IX, ry = threadIdx.x / IX;
  const bool last = a.j == a.J - 1;
  uint32_t keep = 0;
#pragma unroll 1
  for (int c = 0; c < CH; ++c) {
    float cn[IQ];
    smooth_tile<D>(A, Bv, c, ry, rx, cn);
    const float q = MODE == WAVE_ITERATE ? (c == 1 ? sbl : sbl * mu) : 1.f;
#pragma unroll
    for (int k = 0; k < IQ; ++k) {
      const int r = ry + k * (INT / IX);
      const int yy = y0 + r, xx = x0 + rx;
      if (yy >= n || xx >= n) continue;
      const float cj = A[(c * G::AY + r + 2 * D) * G::PITCH + rx + 2 * D];
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
          const uint32_t bit = 1u << (2 * k + s);
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
  }
}

template <int CH, int MODE, int D>
__global__ void __launch_bounds__(INT) k_iuwt_syn(IuwtArgs a) {
  using G = Geo<D>;
  extern __shared__ float ism[];
  float *A = ism;
  float *Bv = A + CH * G::AY * G::PITCH;
  const int n = a.n;
  const int ntx = (n + IX - 1) / IX;
  const int x0 = (blockIdx.x % ntx) * IX, y0 = (blockIdx.x / ntx) * IY;
  const int l = blockIdx.y;
  const size_t NN = (size_t)n * n, CS = (size_t)a.L * NN;
  load_tile<CH, D, false, MODE>(a, A, y0, x0, l, 0.f);
  __syncthreads();
  const int rx = threadIdx.x % IX, ry = threadIdx.x / IX;
  float o[CH][IQ];
#pragma unroll 1
  for (int c = 0; c < CH; ++c) {
    float sr[IQ];
    smooth_tile<D>(A, Bv, c, ry, rx, sr);
#pragma unroll
    for (int k = 0; k < IQ; ++k) {
      const int yy = y0 + ry + k * (INT / IX), xx = x0 + rx;
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
  }
  if (a.j > 0) return;
  const float mu = (MODE == WAVE_ITERATE) ? (float)a.sc[l / a.Lc].mu : 0.f;
  const float tau = (MODE == WAVE_ITERATE) ? (float)a.sc[l / a.Lc].tau : 0.f;
  const float bl = (MODE == WAVE_ITERATE) ? a.beta[l] : 0.f;
#pragma unroll
  for (int k = 0; k < IQ; ++k) {
    const int yy = y0 + ry + k * (INT / IX), xx = x0 + rx;
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

template <int CH, int MODE, int D>
cudaError_t launch_ana_d(const IuwtArgs &a, int L, int n, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_iuwt_ana<CH, MODE, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)iuwt_smem<D>(CH));
    attr = true;
  }
  k_iuwt_ana<CH, MODE, D><<<dim3(itiles(n), L), INT, iuwt_smem<D>(CH), st>>>(a);
  return cudaGetLastError();
}

template <int CH, int MODE, int D>
cudaError_t launch_syn_d(const IuwtArgs &a, int L, int n, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_iuwt_syn<CH, MODE, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)iuwt_smem<D>(CH));
    attr = true;
  }
  k_iuwt_syn<CH, MODE, D><<<dim3(itiles(n), L), INT, iuwt_smem<D>(CH), st>>>(a);
  return cudaGetLastError();
}

template <int CH, int MODE>
cudaError_t ana_all(const WaveArgs &w, IuwtArgs a, cudaStream_t st) {
  const double vox = (double)CH * w.L * w.n * w.n;
  for (int j = 0; j < w.J; ++j) {
    a.j = j;
    const double bytes = vox * ((j == 0 && MODE == WAVE_ITERATE ? 8.0 : 4.0) +
                                (MODE == WAVE_ITERATE ? 8.0 : 4.0) * (j == w.J - 1 ? 2 : 1) +
                                (j == w.J - 1 ? 0.0 : 4.0));
    ProfScope ps(w.prof, "iuwt_ana_dual", bytes, vox * 22.0, st);
    cudaError_t e;
    switch (j) {
      case 0: e = launch_ana_d<CH, MODE, 1>(a, w.L, w.n, st); break;
      case 1: e = launch_ana_d<CH, MODE, 2>(a, w.L, w.n, st); break;
      case 2: e = launch_ana_d<CH, MODE, 4>(a, w.L, w.n, st); break;
      default: e = launch_ana_d<CH, MODE, 8>(a, w.L, w.n, st); break;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int CH, int MODE>
cudaError_t syn_all(const WaveArgs &w, IuwtArgs a, cudaStream_t st) {
  const double vox = (double)CH * w.L * w.n * w.n;
  for (int j = w.J - 1; j >= 0; --j) {
    a.j = j;
    const double bytes = vox * ((j == w.J - 1 ? 8.0 : 4.0) + 8.0 * (j > 0) + 4.0 * (j == 0) +
                                (j > 0 ? 4.0 : (MODE == WAVE_ITERATE ? 16.0 : 4.0)));
    ProfScope ps(w.prof, j == 0 ? "iuwt_syn_prox" : "iuwt_syn", bytes, vox * 22.0, st);
    cudaError_t e;
    switch (j) {
      case 0: e = launch_syn_d<CH, MODE, 1>(a, w.L, w.n, st); break;
      case 1: e = launch_syn_d<CH, MODE, 2>(a, w.L, w.n, st); break;
      case 2: e = launch_syn_d<CH, MODE, 4>(a, w.L, w.n, st); break;
      default: e = launch_syn_d<CH, MODE, 8>(a, w.L, w.n, st); break;
    }
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
