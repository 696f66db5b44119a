// Spectral step of Algorithm 2 (eqs. vt, v, upt), run for every pixel n:
//     v~ = v + sigma gamma_n C (2 x~^n - x^n);   v = sat(v~);   t = gamma_n C^T v
// with C the orthonormal L x L DCT-II (Sec. 4.2.1).  Over a tile of PT pixels
// both products are dense [L x L] x [L x PT] contractions, run on the tensor
// cores as 3xTF32 split products (a_hi b_hi + a_hi b_lo + a_lo b_hi, FP32
// accumulation), which keeps FP32 accuracy.  C is pre-split on the host; the
// B operand is split in registers.
//
// ADA-PT groups (C = 3 chains) reuse the primal's mask Pi(v~) and add the
// inhomogeneous terms of Algorithm 4:
//     v~'_gamma = v'_gamma + sigma alpha_n C (2x~ - x + gamma (2x~' - x'))
//     t'_gamma  = alpha_n C^T (gamma v'_gamma + v)
// while Algorithm 3's spectral step is the homogeneous one.
//
// Layout: every cube is band-major [L][N], so the tile [L x PT] is PT
// consecutive pixels of each band (coalesced rows); the band<->pixel
// "exchange" of the paper's master/slave split becomes this access pattern.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "kernels.h"

namespace muffin {

namespace {

constexpr int DT = 128;   // threads (4 warps)

__device__ __forceinline__ uint32_t to_tf32(float f) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4],
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_wait0() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

struct DctKArgs {
  int n, L, Lp, inverse;
  size_t npix;                // pixels per band (n * n, or a pixel block)
  int ctas_per_sm;            // persistent grid size (0: max resident)
  int B;                      // cubes; blockIdx.y selects the cube
  const float *a1hi, *a1lo;   // first product: C (or C^T for the inverse operator)
  const float *a2hi, *a2lo;   // second product: C^T
  const float *alpha;
  const DevScalars *sc;
  const float *xt, *x;        // iterate inputs [C][L][N]
  float *v, *t;               // iterate state [C][L][N]
  const float *in;            // operator input [L][N]
  float *out;                 // operator output [L][N]
};

// acc[nt][e] (e: c0..c3) = sum_k A[m0 + row(e)][k] * B[k][nt*8 + col(e)]
template <int PT>
__device__ __forceinline__ void tile_gemm(const float *__restrict__ Ahi,
                                          const float *__restrict__ Alo, int Lp,
                                          int m0, const float *B, int PP,
                                          float (&acc)[PT / 8][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < PT / 8; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
  // the A fragments (rows of C from global memory, L2-resident) of the next
  // k-step are requested before the current step's products
  uint32_t nh[4], nl[4];
  auto frag = [&](int k0, uint32_t (&h)[4], uint32_t (&lo)[4]) {
    const int r0 = (m0 + g) * Lp + k0 + t, r1 = (m0 + g + 8) * Lp + k0 + t;
    h[0] = __float_as_uint(__ldg(Ahi + r0));
    h[1] = __float_as_uint(__ldg(Ahi + r1));
    h[2] = __float_as_uint(__ldg(Ahi + r0 + 4));
    h[3] = __float_as_uint(__ldg(Ahi + r1 + 4));
    lo[0] = __float_as_uint(__ldg(Alo + r0));
    lo[1] = __float_as_uint(__ldg(Alo + r1));
    lo[2] = __float_as_uint(__ldg(Alo + r0 + 4));
    lo[3] = __float_as_uint(__ldg(Alo + r1 + 4));
  };
  frag(0, nh, nl);
  for (int k0 = 0; k0 < Lp; k0 += 8) {
    uint32_t ah[4], al[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { ah[q] = nh[q]; al[q] = nl[q]; }
    if (k0 + 8 < Lp) frag(k0 + 8, nh, nl);
    const float *b0p = B + (k0 + t) * PP + g;
    const float *b1p = B + (k0 + t + 4) * PP + g;
#pragma unroll
    for (int nt = 0; nt < PT / 8; ++nt) {
      const float f0 = b0p[nt * 8], f1 = b1p[nt * 8];
      const uint32_t h0 = to_tf32(f0), h1 = to_tf32(f1);
      const uint32_t l0 = to_tf32(f0 - __uint_as_float(h0));
      const uint32_t l1 = to_tf32(f1 - __uint_as_float(h1));
      mma_tf32(acc[nt], al, h0, h1);
      mma_tf32(acc[nt], ah, l0, l1);
      mma_tf32(acc[nt], ah, h0, h1);
    }
  }
}

// tile_gemm with A in shared memory ([Lp][CP], TF32 hi/lo halves of C):
// TR = false multiplies by C, TR = true by C^T (transposed indexing)
template <int PT, bool TR>
__device__ __forceinline__ void tile_gemm_s(const float *Ahi, const float *Alo, int CP,
                                            int Lp, int m0, const float *B, int PP,
                                            float (&acc)[PT / 8][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < PT / 8; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
  for (int k0 = 0; k0 < Lp; k0 += 8) {
    uint32_t ah[4], al[4];
    // fragment element (row, col): row m0 + g (+8), col k0 + t (+4)
    int o[4];
    if (!TR) {
      o[0] = (m0 + g) * CP + k0 + t;   o[1] = (m0 + g + 8) * CP + k0 + t;
      o[2] = o[0] + 4;                 o[3] = o[1] + 4;
    } else {
      o[0] = (k0 + t) * CP + m0 + g;   o[1] = o[0] + 8;
      o[2] = o[0] + 4 * CP;            o[3] = o[2] + 8;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ah[q] = __float_as_uint(Ahi[o[q]]);
      al[q] = __float_as_uint(Alo[o[q]]);
    }
    const float *b0p = B + (k0 + t) * PP + g;
    const float *b1p = B + (k0 + t + 4) * PP + g;
#pragma unroll
    for (int nt = 0; nt < PT / 8; ++nt) {
      const float f0 = b0p[nt * 8], f1 = b1p[nt * 8];
      const uint32_t h0 = to_tf32(f0), h1 = to_tf32(f1);
      const uint32_t l0 = to_tf32(f0 - __uint_as_float(h0));
      const uint32_t l1 = to_tf32(f1 - __uint_as_float(h1));
      mma_tf32(acc[nt], al, h0, h1);
      mma_tf32(acc[nt], ah, l0, l1);
      mma_tf32(acc[nt], ah, h0, h1);
    }
  }
}

// rows [0, L) of a [Lp][PT + 8] shared tile -> dst[l * N + n0 + p] with
// 16-byte stores (guarded scalar stores for a ragged last tile)
template <int PT>
__device__ __forceinline__ void store_rows(const float *src, float *dst, int L, int Lp,
                                           size_t N, size_t n0, bool full) {
  constexpr int PP = PT + 8, Q = PT / 4;
  for (int it = threadIdx.x; it < Lp * Q; it += DT) {
    const int l = it / Q, p4 = (it - l * Q) * 4;
    if (l >= L) continue;
    const float *s = src + l * PP + p4;
    float *d = dst + (size_t)l * N + n0 + p4;
    if (full) {
      *reinterpret_cast<float4 *>(d) = *reinterpret_cast<const float4 *>(s);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (n0 + p4 + e < N) d[e] = s[e];
    }
  }
}

// NTHR threads: one warp per 16-band m-tile of C where L allows (256
// bands: 16 warps), so the products of a tile run in parallel
// ALIAS (one chain, at most one m-tile per warp): the new duals stay in
// registers until every warp has finished the first product, then overwrite
// the input tile, so one [Lp][PT + 8] buffer serves both products and the
// pixel tile can be twice as wide (half the L2 reads of C per pixel)
template <int CH, int MODE, int PT, int NTHR, bool ALIAS = false>
__global__ void __launch_bounds__(NTHR) k_dct(DctKArgs a) {
  static_assert(!ALIAS || CH == 1, "the aliased tile holds one chain");
  extern __shared__ float sm[];
  constexpr int PP = PT + 8;
  const int Lp = a.Lp, L = a.L;
  float *zin = sm;                                  // [CH][Lp][PP]
  float *vo = ALIAS ? zin : zin + CH * Lp * PP;     // [CH][Lp][PP]
  float vkeep[ALIAS ? PT / 8 : 1][4];
  int mt_own = -1;
  const size_t N = a.npix;
  const size_t CS = (size_t)a.B * L * N;     // chain stride
  const size_t n0 = (size_t)blockIdx.x * PT;
  const int cube = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const float gamma = (MODE == WAVE_ITERATE) ? (float)a.sc[cube].gamma : 0.f;
  const float sigma = (MODE == WAVE_ITERATE) ? (float)a.sc[cube].sigma : 0.f;
  const size_t cb = (size_t)cube * L * N;    // the cube's first band
  const float *__restrict__ alpha = a.alpha + (size_t)cube * N;

  // loads of several rounds in flight before their first use
#pragma unroll 8
  for (int it = threadIdx.x; it < Lp * PT; it += NTHR) {
    const int l = it / PT, p = it - l * PT;
    const size_t pix = n0 + p;
    const bool ok = l < L && pix < N;
    const size_t j = cb + (size_t)l * N + pix;
    float z[CH];
    if (MODE == WAVE_TRANSFORM) {
      z[0] = ok ? a.in[j] : 0.f;
    } else {
#pragma unroll
      for (int c = 0; c < CH; ++c) z[c] = ok ? 2.f * a.xt[c * CS + j] - a.x[c * CS + j] : 0.f;
      if (CH == 3) z[2] = fmaf(gamma, z[2], z[0]);   // Algorithm 4 input
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) zin[(c * Lp + l) * PP + p] = z[c];
  }
  __syncthreads();

  const int nmt = Lp >> 4;
  for (int mt = warp; mt < nmt; mt += NTHR / 32) {
    uint32_t mask = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      float acc[PT / 8][4];
      tile_gemm<PT>(a.a1hi, a.a1lo, Lp, mt * 16, zin + c * Lp * PP, PP, acc);
#pragma unroll
      for (int nt = 0; nt < PT / 8; ++nt) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = mt * 16 + g + (e >= 2 ? 8 : 0);
          const int p = nt * 8 + 2 * t + (e & 1);
          const size_t pix = n0 + p;
          const bool valid = k < L && pix < N;
          const size_t j = cb + (size_t)k * N + pix;
          if (MODE == WAVE_TRANSFORM) {
            if (valid) a.out[j] = acc[nt][e];
            continue;
          }
          float vn = 0.f;
          if (valid) {
            const float al = alpha[pix];
            const float s1 = (c == 2) ? sigma * al : sigma * gamma * al;
            const float vt = fmaf(s1, acc[nt][e], a.v[c * CS + j]);
            if (c == 0) {
              vn = satf(vt);
              if (fabsf(vt) <= 1.f) mask |= 1u << (nt * 4 + e);
            } else {
              vn = ((mask >> (nt * 4 + e)) & 1u) ? vt : 0.f;
            }
            a.v[c * CS + j] = vn;
          }
          if constexpr (ALIAS) vkeep[nt][e] = vn;
          else vo[(c * Lp + k) * PP + p] = vn;
        }
      }
    }
    if constexpr (ALIAS) mt_own = mt;
  }
  if (MODE == WAVE_TRANSFORM) return;
  __syncthreads();
  if constexpr (ALIAS) {
    if (mt_own >= 0) {
#pragma unroll
      for (int nt = 0; nt < PT / 8; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = mt_own * 16 + g + (e >= 2 ? 8 : 0);
          vo[k * PP + nt * 8 + 2 * t + (e & 1)] = vkeep[nt][e];
        }
    }
    __syncthreads();
  }
  if (CH == 3) {
    for (int it = threadIdx.x; it < Lp * PT; it += NTHR) {
      const int l = it / PT, p = it - l * PT;
      float *d = vo + (2 * Lp + l) * PP + p;
      *d = fmaf(gamma, *d, vo[l * PP + p]);     // gamma v'_gamma + v
    }
    __syncthreads();
  }
  for (int mt = warp; mt < nmt; mt += NTHR / 32) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      float acc[PT / 8][4];
      tile_gemm<PT>(a.a2hi, a.a2lo, Lp, mt * 16, vo + c * Lp * PP, PP, acc);
#pragma unroll
      for (int nt = 0; nt < PT / 8; ++nt) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int l = mt * 16 + g + (e >= 2 ? 8 : 0);
          const int p = nt * 8 + 2 * t + (e & 1);
          const size_t pix = n0 + p;
          if (l < L && pix < N) {
            const float al = alpha[pix];
            const float s2 = (c == 2) ? al : gamma * al;
            a.t[c * CS + cb + (size_t)l * N + pix] = s2 * acc[nt][e];
          }
        }
      }
    }
  }
}

// Iteration kernel for L <= 64 (one 16-row m-tile per warp).  Persistent:
// each CTA copies the TF32 hi/lo halves of C into shared memory once and
// then walks pixel tiles, so the A fragments of both products come from
// shared memory (C^T by transposed indexing).  Global traffic is coalesced:
// the input tile is read with 16-byte loads, each chain's old duals arrive
// by cp.async while the chain's first product runs, and the new duals and
// t are staged in shared memory and written back as whole 128-byte rows.
template <int CH, int PT>
__global__ void __launch_bounds__(DT, 3) k_dct_small(DctKArgs a) {
  extern __shared__ float sm[];
  constexpr int PP = PT + 8;
  constexpr int Q = PT / 4;               // float4 per tile row
  const int Lp = a.Lp, L = a.L, CP = a.Lp + 4;
  float *chs = sm;                        // [Lp][CP] C, TF32 high part
  float *cls = chs + Lp * CP;             // [Lp][CP] C, TF32 low part
  float *zb = cls + Lp * CP;              // [CH][Lp][PP] products' B operands
  float *vb = zb + CH * Lp * PP;          // [Lp][PP] old duals / t staging
  float *als = vb + Lp * PP;              // [PT] alpha of the tile
  const size_t N = a.npix;
  const size_t CS = (size_t)a.B * L * N;  // chain stride
  const int tpc = (int)((N + PT - 1) / PT);
  const int ntiles = tpc * a.B;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int mt = warp;
  const bool has = mt * 16 < Lp;
  for (int it = threadIdx.x; it < Lp * Lp; it += DT) {
    const int r = it / Lp, c = it - r * Lp;
    chs[r * CP + c] = a.a1hi[it];
    cls[r * CP + c] = a.a1lo[it];
  }
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int cube = tile / tpc;
    const size_t n0 = (size_t)(tile - cube * tpc) * PT;
    const float gamma = (float)a.sc[cube].gamma;
    const float sigma = (float)a.sc[cube].sigma;
    const size_t cb = (size_t)cube * L * N;    // the cube's first band
    const bool full = n0 + PT <= N;
    __syncthreads();                           // previous tile done with zb, vb, als
    for (int it = threadIdx.x; it < Lp * Q; it += DT) {
      const int l = it / Q, p4 = (it - l * Q) * 4;
      float z[CH][4];
      if (l < L && full) {
        const size_t j = cb + (size_t)l * N + n0 + p4;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const float4 xt = *reinterpret_cast<const float4 *>(a.xt + c * CS + j);
          const float4 xx = *reinterpret_cast<const float4 *>(a.x + c * CS + j);
          z[c][0] = 2.f * xt.x - xx.x; z[c][1] = 2.f * xt.y - xx.y;
          z[c][2] = 2.f * xt.z - xx.z; z[c][3] = 2.f * xt.w - xx.w;
        }
      } else {
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const size_t pix = n0 + p4 + e;
            const size_t j = cb + (size_t)l * N + pix;
            z[c][e] = (l < L && pix < N) ? 2.f * a.xt[c * CS + j] - a.x[c * CS + j] : 0.f;
          }
      }
      if (CH == 3)
#pragma unroll
        for (int e = 0; e < 4; ++e) z[2][e] = fmaf(gamma, z[2][e], z[0][e]);  // Algorithm 4
#pragma unroll
      for (int c = 0; c < CH; ++c)
        *reinterpret_cast<float4 *>(zb + (c * Lp + l) * PP + p4) =
            make_float4(z[c][0], z[c][1], z[c][2], z[c][3]);
    }
    for (int it = threadIdx.x; it < PT; it += DT)
      als[it] = n0 + it < N ? a.alpha[(size_t)cube * N + n0 + it] : 0.f;
    // first product and dual update, one chain at a time
    uint32_t keep = 0;
#pragma unroll 1
    for (int c = 0; c < CH; ++c) {
      // vb is free: the barrier after the previous chain's epilogue
      for (int it = threadIdx.x; it < Lp * Q; it += DT) {
        const int l = it / Q, p4 = (it - l * Q) * 4;
        float *d = vb + l * PP + p4;
        const size_t j = c * CS + cb + (size_t)l * N + n0 + p4;
        if (l < L && full) {
          cp_async16(d, a.v + j);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) d[e] = (l < L && n0 + p4 + e < N) ? a.v[j + e] : 0.f;
        }
      }
      cp_commit();
      if (c == 0) __syncthreads();             // the input tile and alpha are in place
      float acc[PT / 8][4];
      if (has) tile_gemm_s<PT, false>(chs, cls, CP, Lp, mt * 16, zb + c * Lp * PP, PP, acc);
      cp_wait0();
      __syncthreads();                         // vb landed; every warp has read zb[c]
      if (has) {
        const float sg = c == 2 ? sigma : sigma * gamma;
#pragma unroll
        for (int nt = 0; nt < PT / 8; ++nt)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int k = mt * 16 + g + (e >= 2 ? 8 : 0);
            const int p = nt * 8 + 2 * t + (e & 1);
            float vn = 0.f;
            if (k < L && n0 + p < N) {
              const float vt = fmaf(sg * als[p], acc[nt][e], vb[k * PP + p]);
              const uint32_t bit = 1u << (nt * 4 + e);
              if (c == 0) {
                vn = satf(vt);
                if (fabsf(vt) <= 1.f) keep |= bit;
              } else {
                vn = (keep & bit) ? vt : 0.f;
              }
            }
            zb[(c * Lp + k) * PP + p] = vn;
          }
      }
      __syncthreads();
      store_rows<PT>(zb + c * Lp * PP, a.v + c * CS + cb, L, Lp, N, n0, full);
    }
    if (CH == 3) {
      __syncthreads();                         // the stores above read zb[0], zb[2]
      for (int it = threadIdx.x; it < Lp * PT; it += DT) {
        const int l = it / PT, p = it - l * PT;
        float *d = zb + (2 * Lp + l) * PP + p;
        *d = fmaf(gamma, *d, zb[l * PP + p]);  // gamma v'_gamma + v
      }
    }
    // back-projection t = gamma_n C^T v (per chain scale of Algorithms 3/4)
#pragma unroll 1
    for (int c = 0; c < CH; ++c) {
      __syncthreads();                         // zb[c] final; vb free
      float acc2[PT / 8][4];
      if (has) {
        tile_gemm_s<PT, true>(chs, cls, CP, Lp, mt * 16, zb + c * Lp * PP, PP, acc2);
#pragma unroll
        for (int nt = 0; nt < PT / 8; ++nt)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int l = mt * 16 + g + (e >= 2 ? 8 : 0);
            const int p = nt * 8 + 2 * t + (e & 1);
            const float s2 = (c == 2) ? als[p] : gamma * als[p];
            vb[l * PP + p] = s2 * acc2[nt][e];
          }
      }
      __syncthreads();
      store_rows<PT>(vb, a.t + c * CS + cb, L, Lp, N, n0, full);
    }
  }
}

template <int CH>
cudaError_t launch_dct_small(const DctKArgs &a, cudaStream_t st, Prof *prof) {
  constexpr int PT = 32;
  const size_t sm = ((size_t)2 * a.Lp * (a.Lp + 4) + (size_t)(CH + 1) * a.Lp * (PT + 8) + PT) *
                    sizeof(float);
  static bool attr = false;
  static int per_sm = 0, sms = 0;
  if (!attr) {
    cudaFuncSetAttribute(k_dct_small<CH, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    attr = true;
  }
  static size_t sm_seen = 0;
  if (sm != sm_seen) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dct_small<CH, PT>, DT, sm);
    if (per_sm < 1) per_sm = 1;
    sm_seen = sm;
  }
  const size_t N = a.npix;
  const size_t ntiles = ((N + PT - 1) / PT) * (size_t)a.B;
  const int use = a.ctas_per_sm > 0 ? std::min(a.ctas_per_sm, per_sm) : per_sm;
  const size_t grid = std::min(ntiles, (size_t)use * (size_t)sms);
  const double vox = (double)N * a.L * a.B;
  ProfScope ps(prof, "spectral_dual", CH * vox * 20.0, 2.0 * CH * 2.0 * a.L * vox, st);
  k_dct_small<CH, PT><<<(unsigned)grid, DT, sm, st>>>(a);
  return cudaGetLastError();
}

template <int CH, int MODE, int PT, int NTHR, bool ALIAS = false>
cudaError_t launch_dct_t(const DctKArgs &a, cudaStream_t st, Prof *prof) {
  const size_t sm = (size_t)(ALIAS ? 1 : 2) * CH * a.Lp * (PT + 8) * sizeof(float);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dct<CH, MODE, PT, NTHR, ALIAS>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const size_t N = a.npix;
  const double vox = (double)N * a.L * a.B;
  ProfScope ps(prof, MODE == WAVE_ITERATE ? "spectral_dual" : "spectral_op",
               MODE == WAVE_ITERATE ? CH * vox * 20.0 : vox * 8.0,
               (MODE == WAVE_ITERATE ? 2.0 : 1.0) * CH * 2.0 * a.L * vox, st);
  k_dct<CH, MODE, PT, NTHR, ALIAS><<<dim3((unsigned)((N + PT - 1) / PT), a.B), NTHR, sm, st>>>(a);
  return cudaGetLastError();
}

template <int CH, int MODE, int PT>
cudaError_t launch_dct(const DctKArgs &a, cudaStream_t st, Prof *prof) {
  if (a.Lp >= 256) return launch_dct_t<CH, MODE, PT, 512>(a, st, prof);
  if (a.Lp >= 128) return launch_dct_t<CH, MODE, PT, 256>(a, st, prof);
  return launch_dct_t<CH, MODE, PT, DT>(a, st, prof);
}

template <int CH, int MODE>
cudaError_t launch_dct_pt(const DctKArgs &a, cudaStream_t st, Prof *prof) {
  // largest pixel tile whose two [CH][Lp][PT+8] buffers fit in the shared
  // memory: every tile reads all of C from L2 once per product, so wider
  // tiles cut that traffic per pixel (64 pixels for one chain up to 256
  // bands)
  const size_t per64 = (size_t)2 * CH * a.Lp * 72 * sizeof(float);
  const size_t per32 = (size_t)2 * CH * a.Lp * 40 * sizeof(float);
  // one chain with 129 .. 256 bands: the aliased 128-pixel tile (16 warps,
  // one 16-band tile of C each)
  if (CH == 1 && a.Lp > 128 && a.Lp <= 256)
    return launch_dct_t<1, MODE, 128, 512, true>(a, st, prof);
  if (a.Lp > 64 && per64 <= 200 * 1024) return launch_dct<CH, MODE, 64>(a, st, prof);
  if (per32 <= 160 * 1024) return launch_dct<CH, MODE, 32>(a, st, prof);
  return launch_dct<CH, MODE, 16>(a, st, prof);
}

}  // namespace

cudaError_t dct_dual(const DctArgs &d, const Group &gr, cudaStream_t st) {
  DctKArgs a{};
  a.n = d.n; a.L = d.L; a.Lp = d.Lp; a.B = d.B > 0 ? d.B : 1;
  a.npix = d.npix ? d.npix : (size_t)d.n * d.n;
  a.a1hi = d.chi; a.a1lo = d.clo; a.a2hi = d.cthi; a.a2lo = d.ctlo;
  a.alpha = d.alpha; a.sc = d.sc; a.ctas_per_sm = d.ctas_per_sm;
  a.xt = gr.xt; a.x = gr.x; a.v = gr.v; a.t = gr.t;
  if (d.f32) return dct_dual_f32(d, gr, st);
  if (d.tc && d.L == 64 && d.Lp == 64) return dct_dual_tc(d, gr, d.err, st);
  if (d.Lp <= 64) {
    if (gr.C == 3) return launch_dct_small<3>(a, st, d.prof);
    return launch_dct_small<1>(a, st, d.prof);
  }
  if (gr.C == 3) return launch_dct_pt<3, WAVE_ITERATE>(a, st, d.prof);
  return launch_dct_pt<1, WAVE_ITERATE>(a, st, d.prof);
}

cudaError_t dct_op(const DctArgs &d, const float *in, float *out, int inverse,
                   cudaStream_t st) {
  if (d.f32) return dct_op_f32(d, in, out, inverse, st);
  DctKArgs a{};
  a.n = d.n; a.L = d.L; a.Lp = d.Lp; a.inverse = inverse; a.B = d.B > 0 ? d.B : 1;
  a.npix = d.npix ? d.npix : (size_t)d.n * d.n;
  a.a1hi = inverse ? d.cthi : d.chi;
  a.a1lo = inverse ? d.ctlo : d.clo;
  a.in = in; a.out = out;
  return launch_dct_pt<1, WAVE_TRANSFORM>(a, st, d.prof);
}

}  // namespace muffin
