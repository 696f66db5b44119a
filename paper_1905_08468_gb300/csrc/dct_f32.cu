// Spectral step in FP32 on the CUDA cores (plans created with precision 1).
//
// The same updates as the tensor-core kernels (Alg. 2 eqs. vt, v, upt and the
// derivative forms of Algs. 3/4), with the orthonormal DCT-II of each pixel
// spectrum (W_lambda, Sec. 4.2.1) computed by a fast transform instead of a
// dense L x L product.  Makhoul's reordering (IEEE Trans. ASSP 28(1), 1980)
// turns a length-L DCT-II into one length-L complex DFT:
//   w_m = x_{2m}, w_{L-1-m} = x_{2m+1} (m < L/2),   W = DFT(w),
//   X'_k = sum_n x_n cos(pi k (2n + 1) / 2L) = Re(e^{-i pi k / 2L} W_k),
// and, for real w, X'_{L-k} = -Im(e^{-i pi k / 2L} W_k); backwards
//   W_k = e^{i pi k / 2L} (X'_k - i X'_{L-k})  (X'_L = 0),  w = DFT^-1(W) / L.
// The orthonormal coefficients are X_0 = X'_0 / sqrt(L), X_k = X'_k sqrt(2/L).
// Two pixels share one complex sequence (real and imaginary parts): after
// the forward DFT they are separated with Z_{L-k} = conj of the real parts'
// spectra, and before the inverse their Hermitian spectra are merged, so
// one DFT of length L serves two pixel spectra each way.  The DFTs are the
// shared-memory Stockham transforms of the gradient passes.  The work is
// O(L log L) per pixel, so the step is bound by its HBM traffic at every L.
//
// A CTA owns a tile of PT = 2 NB pixels of one cube.  Phases: load z = 2 x~ -
// x of every band of the tile (float2 pairs of pixels, coalesced along the
// pixels) into the reordered positions; forward DFTs; per (pixel pair, band
// pair {k, L-k}) task: separate, scale, dual update against the old duals in
// HBM (chain 0 records the mask of sat, the derivative chains apply it),
// store the new duals and write the merged inverse input in place; inverse
// DFTs; store t = gamma alpha C^T v (chain 2: alpha C^T (gamma v'_gamma + v)).
#include <cuda_runtime.h>

#include <cmath>

#include "fft32.cuh"
#include "kernels.h"

namespace muffin {

namespace {

constexpr int FT = 256;   // threads per CTA

template <int L>
struct FShape {
  static constexpr int VPT = fft_vpt(L);
  static constexpr int NB0 = FT * VPT / L;            // sequences the DFT threads cover
  static constexpr int NB = NB0 > 128 ? 128 : NB0;    // pixel pairs per tile
  static constexpr int PT = 2 * NB;                   // pixels per tile
  // padded sequence length, odd so that 16 consecutive pairs hit distinct banks
  static constexpr int PITCH = ((L - 1) + (L - 1) / 16 + 1) | 1;
  static constexpr int NTASK = NB * (L / 2);
  static constexpr int TPT = (NTASK + FT - 1) / FT;   // tasks per thread
  static_assert(NB * L / VPT <= FT, "the DFT threads fit in the CTA");
  static_assert(TPT * 4 <= 32, "mask bits of a thread's tasks fit in 32 bits");
};

struct F32Args {
  int L, B;
  size_t npix;
  const float2 *tab;    // [tw_len] DFT stage twiddles, [L] (cos, sin)(pi k / 2L)
  int tw_len;
  const float *alpha;   // [B][npix]
  const DevScalars *sc; // [B]
  const float *xt, *x;  // iteration inputs [C][B][L][npix]
  float *v, *t;         // duals (in/out) and back-projection (out)
  const float *in;      // operator input [B][L][npix]
  float *out;           // operator output
  int inverse;          // operator: 0 C in, 1 C^T in
};

__device__ __forceinline__ float2 ld2(const float *p) {
  return *reinterpret_cast<const float2 *>(p);
}
__device__ __forceinline__ void st2(float *p, float2 v) {
  *reinterpret_cast<float2 *>(p) = v;
}

// position of band l in the reordered sequence
template <int L>
__device__ __forceinline__ int mpos(int l) {
  return (l & 1) ? L - 1 - (l >> 1) : (l >> 1);
}

template <int L, int CH, int MODE>
__global__ void __launch_bounds__(FT, 2) k_dct_f32(F32Args a) {
  using S = FShape<L>;
  constexpr int NB = S::NB, PT = S::PT, PITCH = S::PITCH;
  extern __shared__ float2 fsm[];
  float2 *tw = fsm;                 // DFT stage twiddles
  float2 *mk = tw + a.tw_len;       // (cos, sin)(pi k / 2L)
  float2 *dat = mk + L;             // [CH][NB][PITCH]
  const int tid = threadIdx.x;
  const size_t N = a.npix;
  const size_t CS = (size_t)a.B * L * N;   // chain stride
  const size_t n0 = (size_t)blockIdx.x * PT;
  const int cube = blockIdx.y;
  const size_t cb = (size_t)cube * L * N;
  const bool fwd_op = MODE == WAVE_TRANSFORM && !a.inverse;
  const bool inv_op = MODE == WAVE_TRANSFORM && a.inverse;
  const float gamma = MODE == WAVE_ITERATE ? (float)a.sc[cube].gamma : 0.f;
  const float sigma = MODE == WAVE_ITERATE ? (float)a.sc[cube].sigma : 0.f;
  const float *__restrict__ alpha = a.alpha + (size_t)cube * N;
  const float r1 = rsqrtf((float)L), r2 = sqrtf(2.f / (float)L);   // s_0, s_k
  const float q1 = rsqrtf((float)L), q2 = rsqrtf(2.f * (float)L);  // inverse input scales
  const float rt2 = 1.41421356237309505f, ch4 = 0.70710678118654752f;

  for (int i = tid; i < a.tw_len + L; i += FT) fsm[i] = a.tab[i];

  // ---- z of every band of the tile, reordered
  if (!inv_op) {
    // loads of several rounds in flight before their first use
    constexpr int UNR = CH == 3 ? 3 : 8;
#pragma unroll UNR
    for (int it = tid; it < L * NB; it += FT) {
      const int s = it % NB, l = it / NB;
      const size_t pix = n0 + 2 * s;
      float2 z[CH];
#pragma unroll
      for (int c = 0; c < CH; ++c) z[c] = make_float2(0.f, 0.f);
      if (pix < N) {
        const size_t j = cb + (size_t)l * N + pix;
        if (MODE == WAVE_TRANSFORM) {
          z[0] = ld2(a.in + j);
        } else {
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const float2 xt = ld2(a.xt + c * CS + j), x = ld2(a.x + c * CS + j);
            z[c] = make_float2(2.f * xt.x - x.x, 2.f * xt.y - x.y);
          }
          if (CH == 3)   // Algorithm 4 input: gamma z'_gamma + z
            z[2] = make_float2(fmaf(gamma, z[2].x, z[0].x), fmaf(gamma, z[2].y, z[0].y));
        }
      }
      const int o = s * PITCH + fpad(mpos<L>(l));
#pragma unroll
      for (int c = 0; c < CH; ++c) dat[c * NB * PITCH + o] = z[c];
    }
  }
  // one chain: the old duals and the pixel weights of this thread's tasks,
  // requested now so that their latency is covered by the forward DFT
  // (three chains have no registers to spare for it)
  constexpr bool PREF = MODE == WAVE_ITERATE && CH == 1;
  constexpr int PF = PREF ? S::TPT : 1;
  float2 pv1[PF], pv2[PF], pal[PF];
  if constexpr (PREF) {
#pragma unroll
    for (int r = 0; r < S::TPT; ++r) {
      const int it = tid + r * FT;
      pv1[r] = pv2[r] = pal[r] = make_float2(0.f, 0.f);
      if (it < S::NTASK) {
        const int s = it % NB, kk = it / NB;
        const int k1 = kk, k2 = kk ? L - kk : L / 2;
        const size_t pix = n0 + 2 * s;
        if (pix < N) {
          pv1[r] = ld2(a.v + cb + (size_t)k1 * N + pix);
          pv2[r] = ld2(a.v + cb + (size_t)k2 * N + pix);
          pal[r] = ld2(alpha + pix);
        }
      }
    }
  }
  if (!inv_op) {
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < CH; ++c) fft_inplace<L, false>(dat + c * NB * PITCH, NB, PITCH, tw);
  } else {
    __syncthreads();   // tables
  }

  // ---- per (pixel pair, band pair) tasks
  uint32_t mask = 0;
  float keep0[CH == 3 ? S::TPT : 1][4];
#pragma unroll 1
  for (int c = 0; c < CH; ++c) {
    float2 *d = dat + c * NB * PITCH;
#pragma unroll
    for (int r = 0; r < S::TPT; ++r) {
      const int it = tid + r * FT;
      if (it >= S::NTASK) break;
      const int s = it % NB, kk = it / NB;
      const int k1 = kk, k2 = kk ? L - kk : L / 2;
      const size_t pix = n0 + 2 * s;
      const bool valid = pix < N;
      const float2 w = mk[kk];
      // orthonormal coefficients X[k1], X[k2] of pixels A (.x) and B (.y)
      float2 X1 = make_float2(0.f, 0.f), X2 = X1;
      if (!inv_op) {
        const float2 Z1 = d[s * PITCH + fpad(k1)], Z2 = d[s * PITCH + fpad(k2)];
        if (kk == 0) {
          X1 = make_float2(Z1.x * r1, Z1.y * r1);
          X2 = make_float2(Z2.x * (ch4 * r2), Z2.y * (ch4 * r2));
        } else {
          // halves of the separated spectra V_A[k1], V_B[k1]
          const float ax = Z1.x + Z2.x, ay = Z1.y - Z2.y;
          const float bx = Z1.y + Z2.y, by = Z2.x - Z1.x;
          const float h = 0.5f * r2;
          X1 = make_float2(h * fmaf(w.x, ax, w.y * ay), h * fmaf(w.x, bx, w.y * by));
          X2 = make_float2(h * fmaf(w.y, ax, -w.x * ay), h * fmaf(w.y, bx, -w.x * by));
        }
      }
      float2 Y1, Y2;   // orthonormal inverse input at k1, k2
      if (fwd_op) {
        if (valid) {
          st2(a.out + cb + (size_t)k1 * N + pix, X1);
          st2(a.out + cb + (size_t)k2 * N + pix, X2);
        }
        continue;
      } else if (inv_op) {
        Y1 = valid ? ld2(a.in + cb + (size_t)k1 * N + pix) : make_float2(0.f, 0.f);
        Y2 = valid ? ld2(a.in + cb + (size_t)k2 * N + pix) : make_float2(0.f, 0.f);
      } else {
        float2 al;
        if constexpr (PREF) al = pal[r];
        else al = valid ? ld2(alpha + pix) : make_float2(0.f, 0.f);
        const float sa = (c == 2) ? sigma : sigma * gamma;
        float *v1p = a.v + c * CS + cb + (size_t)k1 * N + pix;
        float *v2p = a.v + c * CS + cb + (size_t)k2 * N + pix;
        float2 o1, o2;
        if constexpr (PREF) {
          o1 = pv1[r];
          o2 = pv2[r];
        } else {
          o1 = valid ? ld2(v1p) : make_float2(0.f, 0.f);
          o2 = valid ? ld2(v2p) : make_float2(0.f, 0.f);
        }
        float vt[4] = {fmaf(sa * al.x, X1.x, o1.x), fmaf(sa * al.y, X1.y, o1.y),
                       fmaf(sa * al.x, X2.x, o2.x), fmaf(sa * al.y, X2.y, o2.y)};
        float vn[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const uint32_t bit = 1u << (r * 4 + e);
          if (c == 0) {
            vn[e] = satf(vt[e]);
            if (fabsf(vt[e]) <= 1.f) mask |= bit;
          } else {
            vn[e] = (mask & bit) ? vt[e] : 0.f;
          }
        }
        if (valid) {
          st2(v1p, make_float2(vn[0], vn[1]));
          st2(v2p, make_float2(vn[2], vn[3]));
        }
        if constexpr (CH == 3) {
          if (c == 0) {
#pragma unroll
            for (int e = 0; e < 4; ++e) keep0[r][e] = vn[e];
          } else if (c == 2) {   // gamma v'_gamma + v
#pragma unroll
            for (int e = 0; e < 4; ++e) vn[e] = fmaf(gamma, vn[e], keep0[r][e]);
          }
        }
        Y1 = make_float2(vn[0], vn[1]);
        Y2 = make_float2(vn[2], vn[3]);
      }
      // merged inverse input W[k1], W[k2] (1/L folded into the scales)
      float2 W1, W2;
      if (kk == 0) {
        W1 = make_float2(Y1.x * q1, Y1.y * q1);
        W2 = make_float2(Y2.x * (rt2 * q2), Y2.y * (rt2 * q2));
      } else {
        const float pa = Y1.x * q2, pb = Y2.x * q2;   // pixel A: X''[k1], X''[k2]
        const float qa = Y1.y * q2, qb = Y2.y * q2;   // pixel B
        const float2 WA = make_float2(fmaf(w.x, pa, w.y * pb), fmaf(w.y, pa, -w.x * pb));
        const float2 WB = make_float2(fmaf(w.x, qa, w.y * qb), fmaf(w.y, qa, -w.x * qb));
        W1 = make_float2(WA.x - WB.y, WA.y + WB.x);
        W2 = make_float2(WA.x + WB.y, WB.x - WA.y);
      }
      d[s * PITCH + fpad(k1)] = W1;
      d[s * PITCH + fpad(k2)] = W2;
    }
  }
  if (fwd_op) return;
  __syncthreads();
#pragma unroll 1
  for (int c = 0; c < CH; ++c) fft_inplace<L, true>(dat + c * NB * PITCH, NB, PITCH, tw);

  // ---- back in band order: t (iteration) or C^T in (operator)
#pragma unroll 4
  for (int it = tid; it < L * NB; it += FT) {
    const int s = it % NB, l = it / NB;
    const size_t pix = n0 + 2 * s;
    if (pix >= N) continue;
    const int o = s * PITCH + fpad(mpos<L>(l));
    const size_t j = cb + (size_t)l * N + pix;
    if (MODE == WAVE_TRANSFORM) {
      st2(a.out + j, dat[o]);
    } else {
      const float2 al = ld2(alpha + pix);
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const float2 val = dat[c * NB * PITCH + o];
        const float s2 = (c == 2) ? 1.f : gamma;
        st2(a.t + c * CS + j, make_float2(s2 * al.x * val.x, s2 * al.y * val.y));
      }
    }
  }
}

template <int L, int CH, int MODE>
cudaError_t launch_f32(const F32Args &a, cudaStream_t st, Prof *prof) {
  using S = FShape<L>;
  const size_t sm = (size_t)(a.tw_len + L + CH * S::NB * S::PITCH) * sizeof(float2);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dct_f32<L, CH, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    attr = true;
  }
  const double vox = (double)a.npix * L * a.B;
  ProfScope ps(prof, MODE == WAVE_ITERATE ? "spectral_dual" : "spectral_op",
               MODE == WAVE_ITERATE ? CH * vox * 20.0 : vox * 8.0,
               (MODE == WAVE_ITERATE ? 2.0 : 1.0) * CH * vox * (2.5 * std::log2((double)L) + 6.0),
               st);
  const unsigned gx = (unsigned)((a.npix + S::PT - 1) / S::PT);
  k_dct_f32<L, CH, MODE><<<dim3(gx, a.B), FT, sm, st>>>(a);
  return cudaGetLastError();
}

template <int CH, int MODE>
cudaError_t dispatch_f32(const F32Args &a, cudaStream_t st, Prof *prof) {
  switch (a.L) {
    case 2: return launch_f32<2, CH, MODE>(a, st, prof);
    case 4: return launch_f32<4, CH, MODE>(a, st, prof);
    case 8: return launch_f32<8, CH, MODE>(a, st, prof);
    case 16: return launch_f32<16, CH, MODE>(a, st, prof);
    case 32: return launch_f32<32, CH, MODE>(a, st, prof);
    case 64: return launch_f32<64, CH, MODE>(a, st, prof);
    case 128: return launch_f32<128, CH, MODE>(a, st, prof);
    case 256: return launch_f32<256, CH, MODE>(a, st, prof);
    case 512: return launch_f32<512, CH, MODE>(a, st, prof);
    case 1024: return launch_f32<1024, CH, MODE>(a, st, prof);
    default: return cudaErrorInvalidValue;
  }
}

F32Args base_args(const DctArgs &d) {
  F32Args a{};
  a.L = d.L; a.B = d.B > 0 ? d.B : 1;
  a.npix = d.npix ? d.npix : (size_t)d.n * d.n;
  a.tab = d.ftab; a.tw_len = d.ftw_len;
  a.alpha = d.alpha; a.sc = d.sc;
  return a;
}

}  // namespace

int dct_f32_table_len(int L) { return fft_table_len(L) + L; }

void dct_f32_tables(int L, float2 *tab) {
  const int tl = fft_table_len(L);
  fft_tables(L, tab);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < L; ++k) {
    const double th = pi * k / (2.0 * L);
    tab[tl + k] = make_float2((float)std::cos(th), (float)std::sin(th));
  }
}

cudaError_t dct_dual_f32(const DctArgs &d, const Group &gr, cudaStream_t st) {
  F32Args a = base_args(d);
  a.xt = gr.xt; a.x = gr.x; a.v = gr.v; a.t = gr.t;
  if (gr.C == 3) return dispatch_f32<3, WAVE_ITERATE>(a, st, d.prof);
  return dispatch_f32<1, WAVE_ITERATE>(a, st, d.prof);
}

cudaError_t dct_op_f32(const DctArgs &d, const float *in, float *out, int inverse,
                       cudaStream_t st) {
  F32Args a = base_args(d);
  a.in = in; a.out = out; a.inverse = inverse;
  return dispatch_f32<1, WAVE_TRANSFORM>(a, st, d.prof);
}

}  // namespace muffin
