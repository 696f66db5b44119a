// Spatial dictionary kernels: the union W_s of K periodised orthonormal
// Daubechies bases (Sec. 4.2.1), J-level Mallat layout, fused with the MUFFIN
// updates that consume them (Algorithm 2 and its derivatives, Algs. 3/4):
//
//   synthesis + primal prox:  s = mu_l W_s^T u ; m = x - tau (grad + s + t);
//                             x~ = (m)_+                    (eqs. adjointspat2,
//                                                             stpm, stpx)
//   analysis + dual update:   p = u + sigma mu_l W_s (2 x~ - x); u = sat(p)
//                                                            (eqs. stpp, stpu)
//
// One level per launch.  A CTA owns a tile of TY x TX coefficients of every
// subband (2TY x 2TX pixels of the level's input) of one band; level 1 keeps
// its input tile in shared memory and runs all K bases on it, so x~ and x are
// read once for the 8 bases; the analysis of coarser levels runs one basis
// per CTA on the approximation left in an LL scratch by the previous level,
// and every synthesis CTA walks all K bases of its tile (so its copy
// pipeline stays full across the bases).  Periodic
// extension is a wrap of the tile's load indices, which also covers levels
// smaller than a filter (the transform stays the exact periodised one).
//
// The analysis filters run on packed pairs (fma.rn.f32x2): the row pass
// filters two image rows at once (the tile is stored as row pairs) and the
// column pass splits each output into its even- and odd-tap halves.  The
// synthesis has two variants with identical sums: the default keeps the
// coefficient layout its cp.async copies deliver and packs both passes over
// the output parity, (x[2k], x[2k+1]) += (h_2s, h_2s+1) * (c, c); the other
// stores the column pass as row pairs and packs the row pass over two rows.
// Filters live in constant memory and every pass keeps a sliding window of
// taps' inputs in registers.
//
// Chains: a launch advances C = 1 (plain) or C = 3 chains {x, dx/dmu,
// dx/dgamma} of one ADA-PT group.  The derivative channels use the masks of
// the primal channel computed in the same thread (U(m) for the prox, Pi(p)
// for the dual) and the inhomogeneous terms of Algorithm 3:
//   analysis input   w1 = (2x~ - x) + mu (2x~' - x'),  scale sigma beta_l
//   synthesis input  u0 + mu u1,                       scale beta_l
// (Algorithm 4 has its inhomogeneous terms in the spectral step).
#include <cuda_runtime.h>

#include "kernels.h"

namespace muffin {

// filters of db1..db8 (taps beyond 2p are zero): h_i, g_i for the synthesis,
// pairs (h_i, h_i), (g_i, g_i) and (h_2s, h_2s+1), (g_2s, g_2s+1) for the
// analysis
__constant__ float c_h[8][16];
__constant__ float c_g[8][16];
__constant__ float2 c_hh[8][16];
__constant__ float2 c_gg[8][16];
__constant__ float2 c_hp[8][8];
__constant__ float2 c_gp[8][8];

namespace {

constexpr int TY = 16, TX = 32, PMAX = 8, NT = 256;
// analysis tiles, in float2 row pairs (rows 2r, 2r+1 of the input)
constexpr int A_RP = TY + PMAX - 1;                  // input row pairs held
constexpr int A_IP = (2 * TX + 2 * PMAX - 2) | 1;    // odd pitch: conflict-free
constexpr int A_LP = TX + 1;                         // row-pass output pitch
constexpr int QX = 4, QY = 2;                        // outputs per thread
// synthesis tiles: a fixed window of coefficients [k0 - 8, k0 + T) in both
// directions (covers the p - 1 <= 7 halo of every basis), 16-byte aligned
constexpr int S_HALO = 8;
constexpr int S_CH = TY + S_HALO;                    // coefficient rows held
constexpr int S_CP = TX + S_HALO;                    // coefficient pitch (x4 aligned)
constexpr int S_LP = (TX + PMAX - 1) | 1;            // column-pass output pitch (float2)
constexpr int QXP = 2, QYP = 2;                      // coefficient positions per thread
constexpr int QXS = 4;                               // scalar synthesis row item

constexpr size_t ana_smem(int ch) {
  return ((size_t)ch * A_RP * A_IP + 2 * A_RP * A_LP) * sizeof(float2);
}
// the U-ring variant of the size-specialised analysis: the three detail
// tiles of the next steps' (basis, chain) arrive by cp.async into a ring of
// shared-memory slots, RING_AHEAD steps ahead of their dual update
constexpr int RING_SLOTS = 3, RING_AHEAD = 2;
constexpr size_t ring_off(int ch) { return (ana_smem(ch) + 15) / 16 * 16; }
constexpr size_t ring_slot_floats() { return (size_t)3 * TY * TX; }
constexpr size_t ana_smem_ring(int ch) {
  return ring_off(ch) + (size_t)RING_SLOTS * ring_slot_floats() * sizeof(float);
}
constexpr size_t syn_smem(int) {
  return (size_t)(8 * S_CH * S_CP) * sizeof(float) + (size_t)(2 * TY * S_LP) * sizeof(float2);
}

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  return __ffma2_rn(a, b, c);
}

struct AnaArgs {
  int n, M, L, K, last;
  int Lc;                       // bands per cube (per-cube scalars sc[l / Lc])
  const float *in;              // level >= 2: LL_{j-1}; level-1 operator: x
  const float *xt, *x;          // level-1 iteration inputs
  float *ll_out;                // LL_j scratch when !last
  float *u;
  const float *beta;
  const DevScalars *sc;
};

struct SynArgs {
  int n, M, L, K, top, positivity;   // M: output side of this level
  int Lc;                            // bands per cube (per-cube scalars sc[l / Lc])
  const float *ll_in;                // LL_j scratch when !top
  const float *u;
  float *ll_out;                     // LL_{j-1} scratch (levels >= 2)
  const float *x, *g, *t;            // level-1 iteration inputs
  float *xt;                         // level-1 iteration output
  float *out;                        // level-1 operator output
  const float *beta;
  const DevScalars *sc;
};

// cp.async helpers (16- and 4-byte copies global -> shared)
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// ------------------------------------------------------------ analysis
template <int CH, int MODE>
__device__ __forceinline__ void ana_emit(const AnaArgs &a, int l, int bb,
                                         int row, int col, const float (&coef)[CH],
                                         const float (&q)[CH]) {
  const size_t NN = (size_t)a.n * a.n;
  const size_t off = (size_t)row * a.n + col;
  float *u0 = a.u + ((size_t)l * a.K + bb) * NN + off;
  if (MODE == WAVE_TRANSFORM) {
    *u0 = coef[0];
  } else {
    const float p0 = fmaf(q[0], coef[0], *u0);
    *u0 = satf(p0);
    const bool keep = fabsf(p0) <= 1.0f;
#pragma unroll
    for (int c = 1; c < CH; ++c) {
      float *uc = u0 + (size_t)c * a.L * a.K * NN;
      const float pc = fmaf(q[c], coef[c], *uc);
      *uc = keep ? pc : 0.0f;
    }
  }
}

// One (basis, chain) step of an analysis level is split into
//   row pass:  rows of the resident input tile -> lo/hi (shared), item =
//              (row pair, QX outputs); (lo_2r, lo_2r+1) accumulate
//              (h_i, h_i) * (in_2r, in_2r+1), so the result is already the
//              row pair the column pass reads;
//   column pass + dual update: the thread's own item (TY/QY x TX items ==
//              NT threads), four subbands of QY coefficients; out = sum_s
//              (h_2s, h_2s+1) . (lo_2(k+s), lo_2(k+s)+1), the even and odd
//              taps summed in the two lanes.
// The U values a step updates are requested before its row pass so their
// latency overlaps the filtering.  Channel 0 records the mask Pi(p) of each
// output in `keep`; derivative channels (c > 0) apply it.
template <int P>
__device__ __forceinline__ void ana_rows(const float2 *in_c, float2 *lo_s, float2 *hi_s) {
  constexpr int RP = TY + P - 1;
  constexpr int NSX = TX / QX;
  constexpr int NV = 2 * QX + 2 * P - 2;
  for (int it = threadIdx.x; it < RP * NSX; it += NT) {
    const int rp = it % RP, sx = it / RP;
    const float2 *src = in_c + rp * A_IP + 2 * QX * sx;
    float2 v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = src[i];
#pragma unroll
    for (int qq = 0; qq < QX; ++qq) {
      float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < 2 * P; ++i) {
        lo = ffma2(c_hh[P - 1][i], v[2 * qq + i], lo);
        hi = ffma2(c_gg[P - 1][i], v[2 * qq + i], hi);
      }
      lo_s[rp * A_LP + QX * sx + qq] = lo;
      hi_s[rp * A_LP + QX * sx + qq] = hi;
    }
  }
}

__device__ __forceinline__ void ana_rows_dispatch(int p, const float2 *in_c, float2 *lo_s,
                                                  float2 *hi_s) {
  switch (p) {
    case 1: ana_rows<1>(in_c, lo_s, hi_s); break;
    case 2: ana_rows<2>(in_c, lo_s, hi_s); break;
    case 3: ana_rows<3>(in_c, lo_s, hi_s); break;
    case 4: ana_rows<4>(in_c, lo_s, hi_s); break;
    case 5: ana_rows<5>(in_c, lo_s, hi_s); break;
    case 6: ana_rows<6>(in_c, lo_s, hi_s); break;
    case 7: ana_rows<7>(in_c, lo_s, hi_s); break;
    default: ana_rows<8>(in_c, lo_s, hi_s); break;
  }
}

template <int P>
__device__ __forceinline__ void ana_cols(const float2 *lo_s, const float2 *hi_s,
                                         float (&cf)[4][QY]) {
  constexpr int NW = QY + P - 1;
  const int kx = threadIdx.x % TX, s = threadIdx.x / TX;
  const float2 *pl = lo_s + (QY * s) * A_LP + kx;
  const float2 *ph = hi_s + (QY * s) * A_LP + kx;
  float2 vl[NW], vh[NW];
#pragma unroll
  for (int i = 0; i < NW; ++i) { vl[i] = pl[i * A_LP]; vh[i] = ph[i * A_LP]; }
#pragma unroll
  for (int qq = 0; qq < QY; ++qq) {
    float2 ll = make_float2(0.f, 0.f), dy = ll, dx = ll, hh = ll;
#pragma unroll
    for (int j = 0; j < P; ++j) {
      ll = ffma2(c_hp[P - 1][j], vl[qq + j], ll);
      dy = ffma2(c_gp[P - 1][j], vl[qq + j], dy);
      dx = ffma2(c_hp[P - 1][j], vh[qq + j], dx);
      hh = ffma2(c_gp[P - 1][j], vh[qq + j], hh);
    }
    cf[0][qq] = dx.x + dx.y; cf[1][qq] = dy.x + dy.y;
    cf[2][qq] = hh.x + hh.y; cf[3][qq] = ll.x + ll.y;
  }
}

__device__ __forceinline__ void ana_cols_dispatch(int p, const float2 *lo_s,
                                                  const float2 *hi_s, float (&cf)[4][QY]) {
  switch (p) {
    case 1: ana_cols<1>(lo_s, hi_s, cf); break;
    case 2: ana_cols<2>(lo_s, hi_s, cf); break;
    case 3: ana_cols<3>(lo_s, hi_s, cf); break;
    case 4: ana_cols<4>(lo_s, hi_s, cf); break;
    case 5: ana_cols<5>(lo_s, hi_s, cf); break;
    case 6: ana_cols<6>(lo_s, hi_s, cf); break;
    case 7: ana_cols<7>(lo_s, hi_s, cf); break;
    default: ana_cols<8>(lo_s, hi_s, cf); break;
  }
}

// U values the thread's column item updates in step (bb, c): subbands DX
// (low y, high x), DY, HH and, at the last level, LL
template <int MODE, int NS, int MS>
__device__ __forceinline__ void ana_prefetch(const AnaArgs &a, int l, int bb, int c,
                                             int kx0, int ky0, float (&pre)[4][QY]) {
  const int n = NS ? NS : a.n, M = MS ? MS : a.M;
  const int h = M >> 1, hn = h * n;
  const int kx = threadIdx.x % TX, s = threadIdx.x / TX;
  const int kxg = kx0 + kx;
  const float *up = a.u + ((size_t)(c * a.L + l) * a.K + bb) * ((size_t)n * n);
#pragma unroll
  for (int qq = 0; qq < QY; ++qq) {
    const int ky = ky0 + QY * s + qq;
    const int o = ky * n + kxg;
    const bool act = MODE == WAVE_ITERATE && ky < h && kxg < h;
    pre[0][qq] = act ? up[o + h] : 0.f;
    pre[1][qq] = act ? up[o + hn] : 0.f;
    pre[2][qq] = act ? up[o + hn + h] : 0.f;
    pre[3][qq] = (act && !NS && a.last) ? up[o] : 0.f;
  }
}

// dual update p = u + q w, u = sat(p) (or the mask of channel 0) and the
// stores of step (bb, c)
template <int MODE, int NS, int MS>
__device__ __forceinline__ void ana_emit_step(const AnaArgs &a, int l, int bb, int c,
                                              int kx0, int ky0, float q,
                                              const float (&cf)[4][QY],
                                              const float (&pre)[4][QY], uint32_t &keep) {
  const int n = NS ? NS : a.n, M = MS ? MS : a.M;
  const int h = M >> 1, hn = h * n;
  const int kx = threadIdx.x % TX, s = threadIdx.x / TX;
  const int kxg = kx0 + kx;
  float *up = a.u + ((size_t)(c * a.L + l) * a.K + bb) * ((size_t)n * n);
  const bool last = !NS && a.last;   // specialised sizes never run the last level
  float *llp = last ? nullptr : a.ll_out + ((size_t)(c * a.L + l) * a.K + bb) * h * h;
  const int sbo[4] = {h, hn, hn + h, 0};
  if (c == 0) keep = 0;
#pragma unroll
  for (int qq = 0; qq < QY; ++qq) {
    const int ky = ky0 + QY * s + qq;
    if (ky >= h || kxg >= h) continue;
    const int o = ky * n + kxg;
    const int nsb = last ? 4 : 3;
#pragma unroll
    for (int sb = 0; sb < 4; ++sb) {
      if (sb >= nsb) break;
      float val;
      if (MODE == WAVE_TRANSFORM) {
        val = cf[sb][qq];
      } else {
        const float p = fmaf(q, cf[sb][qq], pre[sb][qq]);
        const uint32_t bit = 1u << (sb * QY + qq);
        if (c == 0) {
          val = satf(p);
          if (fabsf(p) <= 1.0f) keep |= bit;
        } else {
          val = (keep & bit) ? p : 0.f;
        }
      }
      up[o + sbo[sb]] = val;
    }
    if (!last) llp[ky * h + kxg] = cf[3][qq];
  }
}

// NS, MS > 0: the image side n and the level's input side M fixed at
// compile time (levels 1 and 2 of the common sizes), so every U offset of
// the dual update is an immediate
template <int CH, int MODE, bool LEVEL1, int NS, int MS, bool RING = false>
__global__ void __launch_bounds__(NT, RING ? 3 : 4) k_ana(AnaArgs a) {
  static_assert(!RING || (NS > 0 && MODE == WAVE_ITERATE),
                "the U ring serves the size-specialised iteration kernels (full tiles)");
  extern __shared__ float2 smem2[];
  float2 *in_s = smem2;                     // [CH][A_RP][A_IP] row pairs
  float2 *lohi = in_s + CH * A_RP * A_IP;   // [A_RP][A_LP] lo, then hi
  float *ring = reinterpret_cast<float *>(reinterpret_cast<char *>(smem2) + ring_off(CH));
  const int n = NS ? NS : a.n, M = MS ? MS : a.M;
  const int h = M >> 1;
  const int ntx = (h + TX - 1) / TX;
  const int kx0 = (blockIdx.x % ntx) * TX, ky0 = (blockIdx.x / ntx) * TY;
  const int l = LEVEL1 ? blockIdx.y : blockIdx.y / a.K;
  const int b = LEVEL1 ? 0 : blockIdx.y % a.K;
  const int P = LEVEL1 ? a.K : b + 1;
  const int RP = TY + P - 1, RW = 2 * TX + 2 * P - 2;
  const int Mm = M - 1;
  const size_t NN = (size_t)n * n;
  const size_t CS = (size_t)a.L * NN;   // channel stride of images
  float mu = 0.f, sbl = 1.f;
  if (MODE == WAVE_ITERATE) {
    const DevScalars &S = a.sc[l / a.Lc];
    mu = (float)S.mu;
    sbl = (float)(S.sigma * (double)a.beta[l]);
  }
  // input tile, two items per thread per round so twice the loads are in
  // flight before the first use
  auto load_item = [&](int it, float (&w)[2][CH]) {
    const int rp = it / RW, cc = it - rp * RW;
    const int xx = (2 * kx0 + cc) & Mm;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int yy = (2 * ky0 + 2 * rp + e) & Mm;
      if (LEVEL1) {
        const size_t pix = (size_t)l * NN + (size_t)yy * n + xx;
        if (MODE == WAVE_TRANSFORM) {
          w[e][0] = a.in[pix];
        } else {
          float z[CH];
#pragma unroll
          for (int c = 0; c < CH; ++c)
            z[c] = 2.f * a.xt[c * CS + pix] - a.x[c * CS + pix];
          w[e][0] = z[0];
          if (CH == 3) { w[e][1] = fmaf(mu, z[1], z[0]); w[e][2] = z[2]; }
        }
      } else {
#pragma unroll
        for (int c = 0; c < CH; ++c)
          w[e][c] = a.in[(((size_t)(c * a.L + l) * a.K + b) * M + yy) * M + xx];
      }
    }
  };
  auto store_item = [&](int it, const float (&w)[2][CH]) {
    const int rp = it / RW, cc = it - rp * RW;
#pragma unroll
    for (int c = 0; c < CH; ++c) in_s[(c * A_RP + rp) * A_IP + cc] = make_float2(w[0][c], w[1][c]);
  };
  const int items = RP * RW;
  for (int it = threadIdx.x; it < items; it += 2 * NT) {
    float w0[2][CH], w1[2][CH];
    const bool two = it + NT < items;
    load_item(it, w0);
    if (two) load_item(it + NT, w1);
    store_item(it, w0);
    if (two) store_item(it + NT, w1);
  }
  __syncthreads();
  // (basis, chain) steps: U requests, row pass, column pass + dual update.
  // One lo/hi buffer keeps shared memory at 4 CTAs per SM, which hides the
  // U loads better than software-pipelining the steps with two buffers.
  const int b0 = LEVEL1 ? 0 : b;
  const int nsteps = (LEVEL1 ? a.K : 1) * CH;
  constexpr int LH = A_RP * A_LP;
  uint32_t keep = 0;
  // ring variant: the detail tiles (DX, DY, HH; TY rows of TX coefficients
  // each) of step t go to slot t mod RING_SLOTS, in 16-byte copies
  auto ring_issue = [&](int t) {
    if (RING && t < nsteps) {
      const int bt = b0 + t / CH, ct = t % CH;
      const int hh = M >> 1, hn = hh * n;
      const float *up = a.u + ((size_t)(ct * a.L + l) * a.K + bt) * ((size_t)n * n);
      float *slot = ring + (size_t)(t % RING_SLOTS) * ring_slot_floats();
      for (int it = threadIdx.x; it < 3 * TY * (TX / 4); it += NT) {
        const int sb = it / (TY * (TX / 4)), r = (it / (TX / 4)) % TY, q = it % (TX / 4);
        const int so = sb == 0 ? hh : (sb == 1 ? hn : hn + hh);
        cp_async16(slot + (sb * TY + r) * TX + 4 * q, up + so + (ky0 + r) * n + kx0 + 4 * q);
      }
    }
    if (RING) cp_commit();
  };
  for (int t = 0; t < RING_AHEAD; ++t) ring_issue(t);
#pragma unroll 1
  for (int s = 0; s < nsteps; ++s) {
    const int bb = b0 + s / CH, c = s % CH;
    float pre[4][QY];
    if (RING) ring_issue(s + RING_AHEAD);
    else ana_prefetch<MODE, NS, MS>(a, l, bb, c, kx0, ky0, pre);
    ana_rows_dispatch(bb + 1, in_s + c * A_RP * A_IP, lohi, lohi + LH);
    if (RING) {
      cp_wait<RING_AHEAD>();        // this step's tiles are in (other threads': barrier)
      __syncthreads();
      const float *slot = ring + (size_t)(s % RING_SLOTS) * ring_slot_floats();
      const int kx = threadIdx.x % TX, sq = threadIdx.x / TX;
#pragma unroll
      for (int qq = 0; qq < QY; ++qq) {
        const int r = QY * sq + qq;
        pre[0][qq] = slot[(0 * TY + r) * TX + kx];
        pre[1][qq] = slot[(1 * TY + r) * TX + kx];
        pre[2][qq] = slot[(2 * TY + r) * TX + kx];
        pre[3][qq] = 0.f;
      }
    } else {
      __syncthreads();
    }
    float cf[4][QY];
    ana_cols_dispatch(bb + 1, lohi, lohi + LH, cf);
    // dual step scale: sigma mu_l (primal, d/dgamma), sigma beta_l (d/dmu)
    const float qc = MODE == WAVE_ITERATE ? (c == 1 ? sbl : sbl * mu) : 1.f;
    ana_emit_step<MODE, NS, MS>(a, l, bb, c, kx0, ky0, qc, cf, pre, keep);
    __syncthreads();
  }
}

// Level-1 analysis + dual update, pipelined: steps run chain-major (chain
// s / K, basis s % K), and one phase holds the row pass of step s and the
// column pass + dual update of step s - 1, with two lo/hi buffers and one
// barrier per step, so the threads that have no row-pass item (short
// filters) go straight to the column work.  Only z0 and one derivative
// chain's input tile are resident (the second tile holds chain 1's input,
// then chain 2's), and chain 0's masks of every basis stay in a 64-bit
// register (8 bits per basis), so shared memory stays at 4 CTAs per SM.  The
// U values of a step are requested one phase ahead.  The row and column
// passes, the inputs and the dual update are k_ana's, so the results are
// bit-identical.  Not the last level (J > 1).
constexpr size_t ana_pipe_smem(int ch) {
  return ((size_t)(ch == 3 ? 2 : 1) * A_RP * A_IP + 4 * A_RP * A_LP) * sizeof(float2);
}

template <int CH, int NS, int MS>
__global__ void __launch_bounds__(NT, 4) k_ana_pipe(AnaArgs a) {
  static_assert(CH == 1 || CH == 3, "one or three chains");
  extern __shared__ float2 smem2[];
  constexpr int TILE = A_RP * A_IP, LH = A_RP * A_LP;
  float2 *in0 = smem2;                           // chain 0: z0
  float2 *in1 = in0 + (CH == 3 ? TILE : 0);      // chain 1, then chain 2
  float2 *lohi = in0 + (CH == 3 ? 2 : 1) * TILE; // [2 buffers][lo, hi]
  const int n = NS ? NS : a.n, M = MS ? MS : a.M;
  const int h = M >> 1;
  const int ntx = (h + TX - 1) / TX;
  const int kx0 = (blockIdx.x % ntx) * TX, ky0 = (blockIdx.x / ntx) * TY;
  const int l = blockIdx.y;
  const int K = a.K;
  const int RP = TY + K - 1, RW = 2 * TX + 2 * K - 2;
  const int Mm = M - 1;
  const size_t NN = (size_t)n * n;
  const size_t CS = (size_t)a.L * NN;
  const DevScalars &S = a.sc[l / a.Lc];
  const float mu = (float)S.mu;
  const float sbl = (float)(S.sigma * (double)a.beta[l]);
  auto zval = [&](int c, size_t pix) { return 2.f * a.xt[c * CS + pix] - a.x[c * CS + pix]; };
  // z0 into in0 and (three chains) z0 + mu z1 into in1
  for (int it = threadIdx.x; it < RP * RW; it += NT) {
    const int rp = it / RW, cc = it - rp * RW;
    const int xx = (2 * kx0 + cc) & Mm;
    float z0[2], w1[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int yy = (2 * ky0 + 2 * rp + e) & Mm;
      const size_t pix = (size_t)l * NN + (size_t)yy * n + xx;
      z0[e] = zval(0, pix);
      if (CH == 3) w1[e] = fmaf(mu, zval(1, pix), z0[e]);
    }
    in0[rp * A_IP + cc] = make_float2(z0[0], z0[1]);
    if (CH == 3) in1[rp * A_IP + cc] = make_float2(w1[0], w1[1]);
  }
  const int nsteps = K * CH;
  uint64_t keep = 0;
  float pre[4][QY];
  ana_prefetch<WAVE_ITERATE, NS, MS>(a, l, 0, 0, kx0, ky0, pre);
  __syncthreads();
#pragma unroll 1
  for (int s = 0; s <= nsteps; ++s) {
    if (CH == 3 && s == 2 * K) {
      // chain 2's input replaces chain 1's (whose last row pass ended before
      // the previous barrier)
      for (int it = threadIdx.x; it < RP * RW; it += NT) {
        const int rp = it / RW, cc = it - rp * RW;
        const int xx = (2 * kx0 + cc) & Mm;
        float z2[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int yy = (2 * ky0 + 2 * rp + e) & Mm;
          z2[e] = zval(2, (size_t)l * NN + (size_t)yy * n + xx);
        }
        in1[rp * A_IP + cc] = make_float2(z2[0], z2[1]);
      }
      __syncthreads();
    }
    if (s < nsteps) {
      const int c = s / K, bb = s - c * K;
      float2 *lh = lohi + (s & 1) * 2 * LH;
      ana_rows_dispatch(bb + 1, c == 0 ? in0 : in1, lh, lh + LH);
    }
    if (s >= 1) {
      const int t = s - 1, c = t / K, bb = t - c * K;
      const float2 *lh = lohi + (t & 1) * 2 * LH;
      float cf[4][QY];
      ana_cols_dispatch(bb + 1, lh, lh + LH, cf);
      // dual step scale: sigma mu_l (primal, d/dgamma), sigma beta_l (d/dmu)
      const float qc = c == 1 ? sbl : sbl * mu;
      uint32_t kb = c == 0 ? 0u : (uint32_t)(keep >> (8 * bb)) & 0xffu;
      ana_emit_step<WAVE_ITERATE, NS, MS>(a, l, bb, c, kx0, ky0, qc, cf, pre, kb);
      if (c == 0) keep |= (uint64_t)kb << (8 * bb);
      if (s < nsteps) {
        const int c2 = s / K;
        ana_prefetch<WAVE_ITERATE, NS, MS>(a, l, s - c2 * K, c2, kx0, ky0, pre);
      }
    }
    if (s < nsteps) __syncthreads();
  }
}

// ------------------------------------------------------------ synthesis
// Inverse of one level: lo/hi along y from (LL, DY) and (DX, HH), then the
// rows.  x[2k+e] = sum_s h[2s+e] a[k-s] + g[2s+e] d[k-s] (transpose of the
// analysis, indices mod the level size).
//
// A CTA walks (chain, basis) steps, chain-major; the coefficient tiles of the
// next step are copied global->shared with cp.async while the current step
// computes (double buffer).  Steps are pure per chain: by linearity the
// d/dmu chain's synthesis of (u + mu u'_mu) (Algorithm 3) is accumulated as
// W^T u + mu W^T u'_mu, continuing from chain 0's finished sum.

constexpr int SUB = S_CH * S_CP;   // one subband tile in shared memory


// copies of the four subband tiles of a (chain, basis) step: rows ky0-8 ..
// ky0+TY-1 and columns kx0-8 .. kx0+TX-1 (mod the level size h).  With
// h >= 8 every aligned group of 4 columns is contiguous in memory (the wrap
// point is a multiple of 4), so whole groups move with 16-byte copies and a
// thread owns at most one group; its offsets are the same in every step and
// are set once.
struct SynSrc {
  int o;          // shared-memory offset of the group in a subband tile (-1: none)
  int ll;         // offset of the LL group in the step's LL source image
  int dy, dx, hh; // offsets of the DY, DX, HH groups in the step's U image
};

__device__ __forceinline__ SynSrc syn_src(const SynArgs &a, int kx0, int ky0) {
  const int h = a.M >> 1, hm = h - 1;
  constexpr int G4 = S_CP / 4;
  SynSrc sr;
  const int it = threadIdx.x;
  if (it >= S_CH * G4) { sr.o = -1; sr.ll = sr.dy = sr.dx = sr.hh = 0; return sr; }
  const int r = it / G4, cc = (it - r * G4) * 4;
  const int ky = (ky0 - S_HALO + r) & hm, kx = (kx0 - S_HALO + cc) & hm;
  sr.o = r * S_CP + cc;
  sr.ll = a.top ? ky * a.n + kx : ky * h + kx;
  sr.dy = (h + ky) * a.n + kx;
  sr.dx = ky * a.n + h + kx;
  sr.hh = (h + ky) * a.n + h + kx;
  return sr;
}
static_assert(S_CH * (S_CP / 4) <= NT, "one 16-byte group per thread");

__device__ __forceinline__ void syn_issue(const SynArgs &a, const SynSrc &sr, float *cf,
                                          int l, int bb, int c) {
  const int h = a.M >> 1, hm = h - 1;
  const size_t NN = (size_t)a.n * a.n;
  const size_t img = (size_t)(c * a.L + l) * a.K + bb;
  const float *up = a.u + img * NN;
  const float *lp = a.top ? up : a.ll_in + img * h * h;
  if (h >= 8) {
    if (sr.o < 0) return;
    cp_async16(cf + sr.o, lp + sr.ll);
    cp_async16(cf + SUB + sr.o, up + sr.dy);
    cp_async16(cf + 2 * SUB + sr.o, up + sr.dx);
    cp_async16(cf + 3 * SUB + sr.o, up + sr.hh);
  } else {
    const int kx0 = 0, ky0 = 0;   // h < 8: a single tile covers the level
    for (int it = threadIdx.x; it < S_CH * S_CP; it += NT) {
      const int r = it / S_CP, cc = it - r * S_CP;
      const int ky = (ky0 - S_HALO + r) & hm, kx = (kx0 - S_HALO + cc) & hm;
      const int o = r * S_CP + cc;
      cp_async4(cf + o, a.top ? up + (size_t)ky * a.n + kx : lp + (size_t)ky * h + kx);
      cp_async4(cf + SUB + o, up + (size_t)(h + ky) * a.n + kx);
      cp_async4(cf + 2 * SUB + o, up + (size_t)ky * a.n + h + kx);
      cp_async4(cf + 3 * SUB + o, up + (size_t)(h + ky) * a.n + h + kx);
    }
  }
}

// one step: column pass into lo/hi, then the thread's row item -> o.
// Column pass (scalar): item = (column, QYP coefficient rows) -> lo/hi of
// the four pixel rows 4j .. 4j+3, stored as row pairs (4j+e, 4j+2+e) so the
// row pass can filter two rows with one packed FMA: (x_r, x_r+2) +=
// (h_i, h_i) * (lo_r, lo_r+2).  The thread's row item is row pair `rp` and
// QXP coefficient positions: o[qq][e] = pixels 2k+e of rows (r, r+2).
template <int P>
__device__ __forceinline__ void syn_step_p(const float *cf, float2 *lo_s, float2 *hi_s,
                                           float2 (&o)[QXP][2]) {
  constexpr int NCOL = TX + P - 1;
  constexpr int NSY = TY / QYP;
  constexpr int NWC = QYP + P - 1;
  constexpr int OFF = S_HALO - (P - 1);     // window offset of this basis' halo
  static_assert(QYP == 2, "a column item covers one row-pair group");
  for (int it = threadIdx.x; it < NSY * NCOL; it += NT) {
    const int kc = it % NCOL, sy = it / NCOL;
    const int base = (QYP * sy + OFF) * S_CP + kc + OFF;
    float vLL[NWC], vDY[NWC], vDX[NWC], vHH[NWC];
#pragma unroll
    for (int i = 0; i < NWC; ++i) {
      vLL[i] = cf[base + i * S_CP];
      vDY[i] = cf[SUB + base + i * S_CP];
      vDX[i] = cf[2 * SUB + base + i * S_CP];
      vHH[i] = cf[3 * SUB + base + i * S_CP];
    }
    float lo[QYP][2], hi[QYP][2];
#pragma unroll
    for (int qq = 0; qq < QYP; ++qq) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        float vl = 0.f, vh = 0.f;
#pragma unroll
        for (int s = 0; s < P; ++s) {
          const int ci = qq + P - 1 - s;
          vl = fmaf(c_h[P - 1][2 * s + e], vLL[ci], vl);
          vl = fmaf(c_g[P - 1][2 * s + e], vDY[ci], vl);
          vh = fmaf(c_h[P - 1][2 * s + e], vDX[ci], vh);
          vh = fmaf(c_g[P - 1][2 * s + e], vHH[ci], vh);
        }
        lo[qq][e] = vl;
        hi[qq][e] = vh;
      }
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      lo_s[(2 * sy + e) * S_LP + kc] = make_float2(lo[0][e], lo[1][e]);
      hi_s[(2 * sy + e) * S_LP + kc] = make_float2(hi[0][e], hi[1][e]);
    }
  }
  __syncthreads();
  constexpr int NWR = QXP + P - 1;
  const int rp = threadIdx.x % TY, sx = threadIdx.x / TY;
  const float2 *pl = lo_s + rp * S_LP + QXP * sx;
  const float2 *ph = hi_s + rp * S_LP + QXP * sx;
  float2 vl[NWR], vh[NWR];
#pragma unroll
  for (int i = 0; i < NWR; ++i) { vl[i] = pl[i]; vh[i] = ph[i]; }
#pragma unroll
  for (int qq = 0; qq < QXP; ++qq) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float2 v = make_float2(0.f, 0.f);
#pragma unroll
      for (int s = 0; s < P; ++s) {
        const int ci = qq + P - 1 - s;
        v = ffma2(c_hh[P - 1][2 * s + e], vl[ci], v);
        v = ffma2(c_gg[P - 1][2 * s + e], vh[ci], v);
      }
      o[qq][e] = v;
    }
  }
}

// Scalar variant of a step: column pass into lo/hi ([2TY][S_LP] floats),
// then the thread's row item: one pixel row, QXS coefficient positions.
template <int P>
__device__ __forceinline__ void syn_step_s(const float *cf, float *lo_s, float *hi_s,
                                           float (&o)[1][2 * QXS]) {
  constexpr int SLP = S_LP;
  constexpr int NSY = TY / QYP;
  constexpr int NWC = QYP + P - 1;
  constexpr int OFF = S_HALO - (P - 1);     // window offset of this basis' halo
  static_assert(NSY * 32 == NT, "one warp per coefficient row group");
  // column item (column kc of the window, coefficient row group sy)
  auto item = [&](int kc, int sy) {
    const int base = (QYP * sy + OFF) * S_CP + kc + OFF;
    // lo (from LL, DY) and hi (from DX, HH) one after the other, so only
    // two coefficient windows are live at a time
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const float *ca = cf + (half ? 2 * SUB : 0) + base;     // LL or DX
      const float *cb = cf + (half ? 3 * SUB : SUB) + base;   // DY or HH
      float *dst = half ? hi_s : lo_s;
      float va[NWC], vb[NWC];
#pragma unroll
      for (int i = 0; i < NWC; ++i) { va[i] = ca[i * S_CP]; vb[i] = cb[i * S_CP]; }
      // both output rows 2k + e of a coefficient row in the lanes of one
      // packed FMA: (h_2s, h_2s+1) * (c, c), same sums in the same order as
      // one scalar FMA per lane
#pragma unroll
      for (int qq = 0; qq < QYP; ++qq) {
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int s = 0; s < P; ++s) {
          const int ci = qq + P - 1 - s;
          v = ffma2(c_hp[P - 1][s], make_float2(va[ci], va[ci]), v);
          v = ffma2(c_gp[P - 1][s], make_float2(vb[ci], vb[ci]), v);
        }
        const int my = 2 * (QYP * sy + qq);
        dst[my * SLP + kc] = v.x;
        dst[(my + 1) * SLP + kc] = v.y;
      }
    }
  };
  // warp w takes row group w and the tile's own TX columns (lane = column,
  // so a warp touches consecutive shared addresses); the P - 1 halo columns
  // of every group follow as a short second round
  item(P - 1 + (threadIdx.x & 31), threadIdx.x >> 5);
  if (P > 1 && threadIdx.x < NSY * (P - 1)) {
    const int sy = threadIdx.x / (P > 1 ? P - 1 : 1);
    item(threadIdx.x - sy * (P - 1), sy);
  }
  __syncthreads();
  constexpr int NWR = QXS + P - 1;
  const int sx = threadIdx.x % (TX / QXS), my = threadIdx.x / (TX / QXS);
  static_assert((TX / QXS) * 2 * TY == NT, "one row item per thread");
  const float *pl = lo_s + my * SLP + QXS * sx;
  const float *ph = hi_s + my * SLP + QXS * sx;
  float vl[NWR], vh[NWR];
#pragma unroll
  for (int i = 0; i < NWR; ++i) { vl[i] = pl[i]; vh[i] = ph[i]; }
#pragma unroll
  for (int qq = 0; qq < QXS; ++qq) {
    float2 v = make_float2(0.f, 0.f);   // pixels 2k, 2k + 1
#pragma unroll
    for (int s = 0; s < P; ++s) {
      const int ci = qq + P - 1 - s;
      v = ffma2(c_hp[P - 1][s], make_float2(vl[ci], vl[ci]), v);
      v = ffma2(c_gp[P - 1][s], make_float2(vh[ci], vh[ci]), v);
    }
    o[0][2 * qq] = v.x;
    o[0][2 * qq + 1] = v.y;
  }
}

// o[ROWS][NO]: the thread's pixels of this step (see k_syn)
template <bool PACKED>
__device__ __forceinline__ void syn_dispatch(int p, const float *cf, float *lo,
                                             float (&o)[PACKED ? 2 : 1][PACKED ? 2 * QXP : 2 * QXS]) {
  if constexpr (PACKED) {
    float2 *lo_s = reinterpret_cast<float2 *>(lo), *hi_s = lo_s + TY * S_LP;
    float2 op[QXP][2];
    switch (p) {
      case 1: syn_step_p<1>(cf, lo_s, hi_s, op); break;
      case 2: syn_step_p<2>(cf, lo_s, hi_s, op); break;
      case 3: syn_step_p<3>(cf, lo_s, hi_s, op); break;
      case 4: syn_step_p<4>(cf, lo_s, hi_s, op); break;
      case 5: syn_step_p<5>(cf, lo_s, hi_s, op); break;
      case 6: syn_step_p<6>(cf, lo_s, hi_s, op); break;
      case 7: syn_step_p<7>(cf, lo_s, hi_s, op); break;
      default: syn_step_p<8>(cf, lo_s, hi_s, op); break;
    }
#pragma unroll
    for (int qq = 0; qq < QXP; ++qq)
#pragma unroll
      for (int e = 0; e < 2; ++e) { o[0][2 * qq + e] = op[qq][e].x; o[1][2 * qq + e] = op[qq][e].y; }
  } else {
    float *lo_s = lo, *hi_s = lo + 2 * TY * S_LP;
    switch (p) {
      case 1: syn_step_s<1>(cf, lo_s, hi_s, o); break;
      case 2: syn_step_s<2>(cf, lo_s, hi_s, o); break;
      case 3: syn_step_s<3>(cf, lo_s, hi_s, o); break;
      case 4: syn_step_s<4>(cf, lo_s, hi_s, o); break;
      case 5: syn_step_s<5>(cf, lo_s, hi_s, o); break;
      case 6: syn_step_s<6>(cf, lo_s, hi_s, o); break;
      case 7: syn_step_s<7>(cf, lo_s, hi_s, o); break;
      default: syn_step_s<8>(cf, lo_s, hi_s, o); break;
    }
  }
}

// PACKED = false: each thread owns one pixel row and 2 QXS pixels;
// PACKED = true: rows r and r + 2 (row pair rp) and 2 QXP pixels each.
// Both variants compute the same sums in the same order (identical results);
// which is faster depends on the shape, so the plan's tuner picks one.
template <int CH, int MODE, bool LEVEL1, bool PACKED>
__global__ void __launch_bounds__(NT, 4) k_syn(SynArgs a) {
  constexpr int ROWS = PACKED ? 2 : 1;   // pixel rows per thread
  constexpr int NO = PACKED ? 2 * QXP : 2 * QXS;   // pixels per row
  extern __shared__ float smem[];
  float *cf0 = smem;                  // two [4][S_CH][S_CP] buffers
  float *lo = smem + 8 * SUB;         // lo/hi of the column pass
  const int h = a.M >> 1;
  const int ntx = (h + TX - 1) / TX;
  const int kx0 = (blockIdx.x % ntx) * TX, ky0 = (blockIdx.x / ntx) * TY;
  const int l = blockIdx.y;
  const float mu = (MODE == WAVE_ITERATE) ? (float)a.sc[l / a.Lc].mu : 0.f;
  int r0, dr, xx0;
  if (PACKED) {
    const int rp = threadIdx.x % TY, sx = threadIdx.x / TY;
    r0 = 4 * (rp >> 1) + (rp & 1); dr = 2; xx0 = 2 * kx0 + NO * sx;
  } else {
    const int sx = threadIdx.x % (TX / QXS), my = threadIdx.x / (TX / QXS);
    r0 = my; dr = 0; xx0 = 2 * kx0 + NO * sx;
  }
  // Steps run chain-major (all bases of chain 0, then chain 1, ...), so a
  // thread holds one running sum: by linearity the d/dmu chain's synthesis
  // of (u + mu u'_mu) is W^T u + mu W^T u'_mu, so chain 1 continues from
  // chain 0's finished sum.  When a chain's last basis is in, its prox runs.
  float sum[ROWS][NO];
#pragma unroll
  for (int j = 0; j < ROWS; ++j)
#pragma unroll
    for (int e = 0; e < NO; ++e) sum[j][e] = 0.f;
  uint32_t keep = 0;                  // chain 0's prox mask, bit j * NO + e
  const size_t NN = (size_t)a.n * a.n;
  const bool own = LEVEL1 && xx0 < a.n;   // the thread has pixels of the level-1 output
  // vector path: the thread's NO pixels of a row are inside it and aligned
  const bool vec = (a.n % NO) == 0 && xx0 + NO <= a.n;
  // chain c's output from its synthesis t: the operator's W^T u, or the
  // primal step x~ = prox(x - tau (grad + scale t + t_spec))
  auto finish = [&](int c, const float (&t)[ROWS][NO]) {
    if (MODE == WAVE_TRANSFORM) {
#pragma unroll
      for (int j = 0; j < ROWS; ++j) {
        const int yy = 2 * ky0 + r0 + dr * j;
        if (yy >= a.n) continue;
        float *dst = a.out + (size_t)l * NN + (size_t)yy * a.n + xx0;
        if (xx0 + NO <= a.n && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
          for (int q = 0; q < NO; q += 4)
            *reinterpret_cast<float4 *>(dst + q) = make_float4(t[j][q], t[j][q + 1], t[j][q + 2], t[j][q + 3]);
        } else {
#pragma unroll
          for (int e = 0; e < NO; ++e)
            if (xx0 + e < a.n) dst[e] = t[j][e];
        }
      }
      return;
    }
    const float tau = (float)a.sc[l / a.Lc].tau;
    const float bl = a.beta[l];
    const size_t CS = (size_t)a.L * NN;
    const float sc = (CH == 3 && c == 1) ? bl : bl * mu;   // mu_l, beta_l, mu_l
#pragma unroll
    for (int j = 0; j < ROWS; ++j) {
      const int yy = 2 * ky0 + r0 + dr * j;
      if (yy >= a.n) continue;
      const size_t i0 = (size_t)l * NN + (size_t)yy * a.n + xx0 + c * CS;
      // four pixels at a time keep the loads' registers few
#pragma unroll
      for (int q = 0; q < NO; q += 4) {
        float xv[4], gv[4], tv[4];
        if (vec) {
          const float4 x4 = *reinterpret_cast<const float4 *>(a.x + i0 + q);
          const float4 g4 = *reinterpret_cast<const float4 *>(a.g + i0 + q);
          const float4 t4 = *reinterpret_cast<const float4 *>(a.t + i0 + q);
          xv[0] = x4.x; xv[1] = x4.y; xv[2] = x4.z; xv[3] = x4.w;
          gv[0] = g4.x; gv[1] = g4.y; gv[2] = g4.z; gv[3] = g4.w;
          tv[0] = t4.x; tv[1] = t4.y; tv[2] = t4.z; tv[3] = t4.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const bool ok = xx0 + q + e < a.n;
            xv[e] = ok ? a.x[i0 + q + e] : 0.f;
            gv[e] = ok ? a.g[i0 + q + e] : 0.f;
            tv[e] = ok ? a.t[i0 + q + e] : 0.f;
          }
        }
        float o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float m = xv[e] - tau * (gv[e] + sc * t[j][q + e] + tv[e]);
          const uint32_t bit = 1u << (j * NO + q + e);
          if (c == 0) {
            const bool k = !a.positivity || m > 0.f;
            if (k) keep |= bit;
            o[e] = k ? m : 0.f;
          } else {
            o[e] = (keep & bit) ? m : 0.f;
          }
        }
        if (vec) {
          *reinterpret_cast<float4 *>(a.xt + i0 + q) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (xx0 + q + e < a.n) a.xt[i0 + q + e] = o[e];
        }
      }
    }
  };
  // (chain, basis) steps; coarser levels write each basis' LL_{j-1}
  const int nsteps = a.K * CH;
  const SynSrc sr = syn_src(a, kx0, ky0);
  syn_issue(a, sr, cf0, l, 0, 0);
  cp_commit();
  // i / K as a multiply-shift (exact for i <= 3K + 1, K <= 8)
  const uint32_t kmag = (65536u + (uint32_t)a.K - 1u) / (uint32_t)a.K;
  for (int i = 0; i < nsteps; ++i) {
    const int c = (int)(((uint32_t)i * kmag) >> 16), bb = i - c * a.K;
    float *cf = cf0 + (i & 1) * 4 * SUB;
    if (i + 1 < nsteps) {
      const int c1 = (int)(((uint32_t)(i + 1) * kmag) >> 16);
      syn_issue(a, sr, cf0 + ((i + 1) & 1) * 4 * SUB, l, i + 1 - c1 * a.K, c1);
      cp_commit();
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    float o[ROWS][NO];
    syn_dispatch<PACKED>(bb + 1, cf, lo, o);
    if (LEVEL1) {
      const float w = (CH == 3 && c == 1) ? mu : 1.f;
#pragma unroll
      for (int j = 0; j < ROWS; ++j)
#pragma unroll
        for (int e = 0; e < NO; ++e) sum[j][e] = fmaf(w, o[j][e], sum[j][e]);
      if (bb == a.K - 1) {                 // chain c is complete
        if (own) finish(c, sum);
        if (!(CH == 3 && c == 0)) {        // chain 1 continues from chain 0's sum
#pragma unroll
          for (int j = 0; j < ROWS; ++j)
#pragma unroll
            for (int e = 0; e < NO; ++e) sum[j][e] = 0.f;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < ROWS; ++j) {
        const int yy = 2 * ky0 + r0 + dr * j;
        if (yy >= a.M) continue;
        float *dst = a.ll_out + (((size_t)(c * a.L + l) * a.K + bb) * a.M + yy) * a.M + xx0;
        if (xx0 + NO <= a.M && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
          for (int q = 0; q < NO; q += 4)
            *reinterpret_cast<float4 *>(dst + q) =
                make_float4(o[j][q], o[j][q + 1], o[j][q + 2], o[j][q + 3]);
        } else {
#pragma unroll
          for (int e = 0; e < NO; ++e)
            if (xx0 + e < a.M) dst[e] = o[j][e];
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ J = 0 (identity bases)
template <int CH, int MODE>
__global__ void k_syn0(SynArgs a) {
  const size_t NN = (size_t)a.n * a.n;
  const size_t tot = (size_t)a.L * NN;
  const size_t US = (size_t)a.L * a.K * NN, CS = (size_t)a.L * NN;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot;
       i += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(i / NN);
    const size_t pix = i - (size_t)l * NN;
    float acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = 0.f;
    const float mu = (MODE == WAVE_ITERATE) ? (float)a.sc[l / a.Lc].mu : 0.f;
    for (int bb = 0; bb < a.K; ++bb) {
      const float *u0 = a.u + ((size_t)l * a.K + bb) * NN + pix;
      float v[CH];
#pragma unroll
      for (int c = 0; c < CH; ++c) v[c] = u0[c * US];
      if (MODE == WAVE_ITERATE && CH == 3) v[1] = fmaf(mu, v[1], v[0]);
#pragma unroll
      for (int c = 0; c < CH; ++c) acc[c] += v[c];
    }
    if (MODE == WAVE_TRANSFORM) { a.out[i] = acc[0]; continue; }
    const float tau = (float)a.sc[l / a.Lc].tau, bl = a.beta[l];
    float sc[CH];
    sc[0] = bl * mu;
    if (CH == 3) { sc[1] = bl; sc[2] = bl * mu; }
    const float m0 = a.x[i] - tau * (a.g[i] + sc[0] * acc[0] + a.t[i]);
    const bool keep = !a.positivity || m0 > 0.f;
    a.xt[i] = keep ? m0 : 0.f;
#pragma unroll
    for (int c = 1; c < CH; ++c) {
      const size_t ic = i + c * CS;
      const float mc = a.x[ic] - tau * (a.g[ic] + sc[c] * acc[c] + a.t[ic]);
      a.xt[ic] = keep ? mc : 0.f;
    }
  }
}

template <int CH, int MODE>
__global__ void k_ana0(AnaArgs a) {
  const size_t NN = (size_t)a.n * a.n;
  const size_t tot = (size_t)a.L * NN, CS = (size_t)a.L * NN;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot;
       i += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(i / NN);
    const size_t pix = i - (size_t)l * NN;
    float w[CH], q[CH];
    if (MODE == WAVE_TRANSFORM) {
      w[0] = a.in[i]; q[0] = 1.f;
    } else {
      const float mu = (float)a.sc[l / a.Lc].mu;
      const float sb = (float)(a.sc[l / a.Lc].sigma * (double)a.beta[l]);
      float z[CH];
#pragma unroll
      for (int c = 0; c < CH; ++c) z[c] = 2.f * a.xt[i + c * CS] - a.x[i + c * CS];
      w[0] = z[0]; q[0] = sb * mu;
      if (CH == 3) { w[1] = fmaf(mu, z[1], z[0]); w[2] = z[2]; q[1] = sb; q[2] = sb * mu; }
    }
    const int row = (int)(pix / a.n), col = (int)(pix % a.n);
    for (int bb = 0; bb < a.K; ++bb) ana_emit<CH, MODE>(a, l, bb, row, col, w, q);
  }
}

// ------------------------------------------------------------ launch helpers
inline int tiles(int h) { return ((h + TX - 1) / TX) * ((h + TY - 1) / TY); }

// algorithmic bytes and flops of one level launch (FP32)
inline double level_flops(int CH, int L, int K, int h) {
  return (double)CH * L * 32.0 * (K * (K + 1) / 2) * (double)h * h;
}

template <int CH, int MODE, bool L1, int NS = 0, int MS = 0, bool RING = false>
cudaError_t launch_ana(const AnaArgs &a, int nblk_y, cudaStream_t st, Prof *prof) {
  const double h = a.M >> 1, rw = MODE == WAVE_ITERATE ? 2.0 : 1.0;
  const double in = L1 ? (double)CH * a.L * a.M * a.M * (MODE == WAVE_ITERATE ? 8.0 : 4.0)
                       : (double)CH * a.L * a.K * a.M * a.M * 4.0;
  const double det = (double)CH * a.L * a.K * 3.0 * h * h * 4.0 * rw;
  const double ll = (double)CH * a.L * a.K * h * h * 4.0 * (a.last ? rw : 1.0);
  ProfScope ps(prof, L1 ? "ana_level1_dual" : "ana_level_dual", in + det + ll,
               level_flops(CH, a.L, L1 ? a.K : a.K, (int)h), st);
  constexpr size_t smem = RING ? ana_smem_ring(CH) : ana_smem(CH);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_ana<CH, MODE, L1, NS, MS, RING>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  k_ana<CH, MODE, L1, NS, MS, RING><<<dim3(tiles(a.M >> 1), nblk_y), NT, smem, st>>>(a);
  return cudaGetLastError();
}

template <int CH, int NS, int MS>
cudaError_t launch_ana_pipe(const AnaArgs &a, int nblk_y, cudaStream_t st, Prof *prof) {
  const double h = a.M >> 1;
  const double in = (double)CH * a.L * a.M * a.M * 8.0;
  const double det = (double)CH * a.L * a.K * 3.0 * h * h * 4.0 * 2.0;
  const double ll = (double)CH * a.L * a.K * h * h * 4.0;
  ProfScope ps(prof, "ana_level1_dual", in + det + ll, level_flops(CH, a.L, a.K, (int)h), st);
  constexpr size_t smem = ana_pipe_smem(CH);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_ana_pipe<CH, NS, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr = true;
  }
  k_ana_pipe<CH, NS, MS><<<dim3(tiles(a.M >> 1), nblk_y), NT, smem, st>>>(a);
  return cudaGetLastError();
}

// the size-specialised analysis launch, with or without the U ring
template <int CH, int MODE, bool L1, int NS, int MS>
cudaError_t launch_ana_sized(const AnaArgs &a, int nblk_y, bool ring, cudaStream_t st,
                             Prof *prof) {
  if constexpr (MODE == WAVE_ITERATE)
    if (ring) return launch_ana<CH, MODE, L1, NS, MS, true>(a, nblk_y, st, prof);
  return launch_ana<CH, MODE, L1, NS, MS, false>(a, nblk_y, st, prof);
}

template <int CH, int MODE, bool L1, bool PACKED>
cudaError_t launch_syn_v(const SynArgs &a, int nblk_y, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_syn<CH, MODE, L1, PACKED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)syn_smem(CH));
    attr = true;
  }
  k_syn<CH, MODE, L1, PACKED><<<dim3(tiles(a.M >> 1), nblk_y), NT, syn_smem(CH), st>>>(a);
  return cudaGetLastError();
}

template <int CH, int MODE, bool L1>
cudaError_t launch_syn(const SynArgs &a, int nblk_y, int packed, cudaStream_t st, Prof *prof) {
  const double h = a.M >> 1;
  const double det = (double)CH * a.L * a.K * 4.0 * h * h * 4.0;   // 3 details + LL
  const double out = L1 ? (double)CH * a.L * a.M * a.M * (MODE == WAVE_ITERATE ? 16.0 : 4.0)
                        : (double)CH * a.L * a.K * a.M * a.M * 4.0;
  ProfScope ps(prof, L1 ? "syn_level1_prox" : "syn_level", det + out,
               level_flops(CH, a.L, a.K, (int)h), st);
  return packed ? launch_syn_v<CH, MODE, L1, true>(a, nblk_y, st)
                : launch_syn_v<CH, MODE, L1, false>(a, nblk_y, st);
}

inline int grid_elem(size_t count) {
  size_t g = (count + 255) / 256;
  return (int)(g > 152 * 16 ? 152 * 16 : (g ? g : 1));
}

template <int CH, int MODE>
cudaError_t synthesis_all(const WaveArgs &w, const SynArgs &base, cudaStream_t st) {
  SynArgs a = base;
  if (w.J == 0) {
    a.M = w.n;
    ProfScope ps(w.prof, "syn_identity_prox", (double)CH * w.L * w.n * w.n * 4.0 * (w.K + 4), 0.0, st);
    k_syn0<CH, MODE><<<grid_elem((size_t)w.L * w.n * w.n), 256, 0, st>>>(a);
    return cudaGetLastError();
  }
  cudaError_t e = cudaSuccess;
  for (int j = w.J; j >= 2; --j) {
    a.M = w.n >> (j - 1);
    a.top = (j == w.J);
    a.ll_in = a.top ? nullptr : w.scratch + w.lvl_off[j];
    a.ll_out = w.scratch + w.lvl_off[j - 1];
    e = launch_syn<CH, MODE, false>(a, w.L, w.syn_packed & 1, st, w.prof);
    if (e != cudaSuccess) return e;
  }
  a.M = w.n;
  a.top = (w.J == 1);
  a.ll_in = a.top ? nullptr : w.scratch + w.lvl_off[1];
  a.ll_out = nullptr;
  return launch_syn<CH, MODE, true>(a, w.L, (w.syn_packed >> 1) & 1, st, w.prof);
}

template <int CH, int MODE>
cudaError_t analysis_all(const WaveArgs &w, const AnaArgs &base, cudaStream_t st) {
  AnaArgs a = base;
  if (w.J == 0) {
    a.M = w.n;
    ProfScope ps(w.prof, "ana_identity_dual", (double)CH * w.L * w.n * w.n * 4.0 * (2 * w.K + 2), 0.0, st);
    k_ana0<CH, MODE><<<grid_elem((size_t)w.L * w.n * w.n), 256, 0, st>>>(a);
    return cudaGetLastError();
  }
  a.M = w.n;
  a.last = (w.J == 1);
  a.ll_out = a.last ? nullptr : w.scratch + w.lvl_off[1];
  // the size-specialised kernels assume a level below (J > level)
  const bool ring = w.ana_ring != 0;
  cudaError_t e = cudaSuccess;
  bool piped = false;
  if constexpr (MODE == WAVE_ITERATE && (CH == 1 || CH == 3)) {
    if (w.ana_pipe && w.J > 1) {
      piped = true;
      e = w.n == 2048 ? launch_ana_pipe<CH, 2048, 2048>(a, w.L, st, w.prof)
          : w.n == 1024 ? launch_ana_pipe<CH, 1024, 1024>(a, w.L, st, w.prof)
          : w.n == 512 ? launch_ana_pipe<CH, 512, 512>(a, w.L, st, w.prof)
                       : launch_ana_pipe<CH, 0, 0>(a, w.L, st, w.prof);
    }
  }
  if (!piped) e = (w.n == 2048 && w.J > 1) ? launch_ana_sized<CH, MODE, true, 2048, 2048>(a, w.L, ring, st, w.prof)
                  : (w.n == 1024 && w.J > 1) ? launch_ana_sized<CH, MODE, true, 1024, 1024>(a, w.L, ring, st, w.prof)
                  : (w.n == 512 && w.J > 1) ? launch_ana_sized<CH, MODE, true, 512, 512>(a, w.L, ring, st, w.prof)
                                            : launch_ana<CH, MODE, true>(a, w.L, st, w.prof);
  for (int j = 2; j <= w.J && e == cudaSuccess; ++j) {
    a.M = w.n >> (j - 1);
    a.in = w.scratch + w.lvl_off[j - 1];
    a.last = (j == w.J);
    a.ll_out = a.last ? nullptr : w.scratch + w.lvl_off[j];
    if (j == 2 && w.J > 2 && w.n == 2048) e = launch_ana_sized<CH, MODE, false, 2048, 1024>(a, w.L * w.K, ring, st, w.prof);
    else if (j == 2 && w.J > 2 && w.n == 1024) e = launch_ana_sized<CH, MODE, false, 1024, 512>(a, w.L * w.K, ring, st, w.prof);
    else if (j == 2 && w.J > 2 && w.n == 512) e = launch_ana_sized<CH, MODE, false, 512, 256>(a, w.L * w.K, ring, st, w.prof);
    else e = launch_ana<CH, MODE, false>(a, w.L * w.K, st, w.prof);
  }
  return e;
}

}  // namespace

cudaError_t upload_filters(const double h[8][16]) {
  float hf[8][16], gf[8][16];
  float2 hh[8][16], gg[8][16], hp[8][8], gp[8][8];
  for (int p = 1; p <= 8; ++p) {
    for (int i = 0; i < 16; ++i) {
      hf[p - 1][i] = i < 2 * p ? (float)h[p - 1][i] : 0.f;
      gf[p - 1][i] = i < 2 * p ? (float)((i & 1 ? -1.0 : 1.0) * h[p - 1][2 * p - 1 - i]) : 0.f;
      hh[p - 1][i] = make_float2(hf[p - 1][i], hf[p - 1][i]);
      gg[p - 1][i] = make_float2(gf[p - 1][i], gf[p - 1][i]);
    }
    for (int j = 0; j < 8; ++j) {
      hp[p - 1][j] = make_float2(hf[p - 1][2 * j], hf[p - 1][2 * j + 1]);
      gp[p - 1][j] = make_float2(gf[p - 1][2 * j], gf[p - 1][2 * j + 1]);
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_h, hf, sizeof(hf));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_g, gf, sizeof(gf));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_hh, hh, sizeof(hh));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_gg, gg, sizeof(gg));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_hp, hp, sizeof(hp));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_gp, gp, sizeof(gp));
  return e;
}

cudaError_t wavelet_synthesis_prox(const WaveArgs &w, const Group &gr,
                                   int positivity, cudaStream_t st) {
  if (w.dict == 1 && w.J > 0) return iuwt_synthesis_prox(w, gr, positivity, st);
  SynArgs a{};
  a.n = w.n; a.L = w.L; a.K = w.K; a.positivity = positivity;
  a.Lc = w.Lc > 0 ? w.Lc : w.L;
  a.u = gr.u; a.x = gr.x; a.g = gr.g; a.t = gr.t; a.xt = gr.xt;
  a.beta = w.beta; a.sc = w.sc;
  if (gr.C == 3) return synthesis_all<3, WAVE_ITERATE>(w, a, st);
  return synthesis_all<1, WAVE_ITERATE>(w, a, st);
}

cudaError_t wavelet_analysis_dual(const WaveArgs &w, const Group &gr,
                                  cudaStream_t st) {
  if (w.dict == 1 && w.J > 0) return iuwt_analysis_dual(w, gr, st);
  AnaArgs a{};
  a.n = w.n; a.L = w.L; a.K = w.K;
  a.Lc = w.Lc > 0 ? w.Lc : w.L;
  a.xt = gr.xt; a.x = gr.x; a.u = gr.u; a.beta = w.beta; a.sc = w.sc;
  if (gr.C == 3) return analysis_all<3, WAVE_ITERATE>(w, a, st);
  return analysis_all<1, WAVE_ITERATE>(w, a, st);
}

cudaError_t wavelet_analysis_op(const WaveArgs &w, const float *x, float *u,
                                cudaStream_t st) {
  if (w.dict == 1 && w.J > 0) return iuwt_analysis_op(w, x, u, st);
  AnaArgs a{};
  a.n = w.n; a.L = w.L; a.K = w.K; a.Lc = w.L; a.in = x; a.u = u;
  return analysis_all<1, WAVE_TRANSFORM>(w, a, st);
}

cudaError_t wavelet_synthesis_op(const WaveArgs &w, const float *u, float *x,
                                 cudaStream_t st) {
  if (w.dict == 1 && w.J > 0) return iuwt_synthesis_op(w, u, x, st);
  SynArgs a{};
  a.n = w.n; a.L = w.L; a.K = w.K; a.Lc = w.L; a.u = u; a.out = x;
  return synthesis_all<1, WAVE_TRANSFORM>(w, a, st);
}

}  // namespace muffin
