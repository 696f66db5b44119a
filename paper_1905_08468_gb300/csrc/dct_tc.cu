// Spectral step of Algorithm 2 (eqs. vt, v, upt) and its derivative forms
// (Algorithms 3/4) for L = 64 bands on the 5th-generation tensor cores:
//     v~ = v + sigma gamma_n C (2 x~^n - x^n);  v = sat(v~);  t = gamma_n C^T v
// over tiles of 128 pixels.  Each product is a [128 x 64] x [64 x 64] TF32
// contraction issued as tcgen05.mma by one thread, three times (a_hi b_hi +
// a_hi b_lo + a_lo b_hi, FP32 accumulation in tensor memory), which keeps
// FP32 accuracy.
//
// Layout: operands sit in shared memory K-major in the canonical
// no-swizzle arrangement of 8-row x 16-byte core matrices (leading byte
// offset 128 B along K, stride byte offset 2 KB along the rows); the TF32
// halves of C (first product) and of C^T (second) stay resident for the
// CTA's lifetime.  A thread owns one pixel and 32 of its 64 bands: it reads
// v and writes v, t as coalesced 128-byte rows (32 consecutive pixels per
// warp and band), splits its row of the A operand into TF32 halves itself,
// and reads its accumulator row straight from tensor memory (the warp's lane
// quadrant), so no shared-memory staging of v or t is needed.  The raw x~
// and x tiles of a chain arrive by 16-byte cp.async into the A buffers
// (free before the split), so the whole 64 KB is in flight at once.
//
// A CTA runs two independent groups of 8 warps that share the C tables but
// own their A tiles, tensor-memory columns (128, or 256 with three chains,
// where the d/dgamma chain accumulates onto chain 0's products) and
// mbarrier, so one group's global traffic overlaps the other's MMAs.  Waits on the mbarriers are
// bounded: on time-out the kernel raises an error flag, waits once more and
// frees its tensor memory; the host turns the flag into MUFFIN_ETIMEOUT.  A
// host-side test hook makes the kernel skip its products so that this path
// runs without any fault.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace muffin {

namespace {

constexpr int TM = 128, TL = 64, KC = TL / 4;   // pixels per tile, bands, core matrices along K
constexpr int GT = 256;                          // threads per group (8 warps)
constexpr int NG = 2;                            // groups per CTA
constexpr int CTA_T = NG * GT;
constexpr uint32_t TILE_B = TM * TL * 4;         // one A tile (32 KB)
constexpr uint32_t CMAT_B = TL * TL * 4;         // one C table (16 KB)
constexpr size_t SMEM = 4 * (size_t)CMAT_B + (size_t)NG * 2 * TILE_B + 1024;
// tensor-memory columns per group: 64 per product accumulator; with three
// chains chain 0's two accumulators are kept for chain 2 (see k_dct_tc)
constexpr uint32_t group_cols(int ch) { return ch == 3 ? 256u : 128u; }
constexpr uint32_t tmem_cols(int ch) { return NG * group_cols(ch); }   // 512 or 256
constexpr long kSpin = 1L << 24;                 // polls of an mbarrier before giving up
constexpr long kSpinInjected = 1L << 12;         // shorter bound when a time-out is injected
// instruction descriptor: D FP32, A and B TF32, both K-major, N = 64, M = 128
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) |
                           ((uint32_t)(TL >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

struct TcArgs {
  int n, L, B;
  size_t npix;                 // pixels per band (n * n, or a pixel block)
  const float *chi, *clo;      // [64][64] C, TF32 high / low part
  const float *cthi, *ctlo;    // [64][64] C^T
  const float *alpha;          // [B][n*n]
  const DevScalars *sc;        // [B]
  const float *xt, *x;         // [C][B*L][n*n]
  float *v, *t;
  int *err;                    // set to 1 when a wait gives up
  int inject;                  // test hook: issue no products, so the waits run out
  long spin;                   // polls of an mbarrier before giving up
};

// byte offset of element (row, k) of a K-major operand with 64 columns
__device__ __forceinline__ uint32_t cm_off(int row, int k) {
  return (uint32_t)(((row >> 3) * KC + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128u >> 4) << 16;                   // leading byte offset (along K)
  d |= (uint64_t)(((uint32_t)KC * 128u) >> 4) << 32;  // stride byte offset (along rows)
  d |= (uint64_t)1 << 46;                             // descriptor version
  return d;                                           // no swizzle, base offset 0
}

__device__ __forceinline__ float tf32r(float f) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
  return __uint_as_float(r);
}

__device__ __forceinline__ void cp16(uint8_t *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

// raw [64 bands][128 pixels] tiles of x~ and x of one chain into stage_a /
// stage_b (16-byte cp.async; zero fill past the last pixel); the caller
// commits, waits and synchronises the group
__device__ __forceinline__ void stage_raw(const float *xt, const float *x, size_t base, size_t N,
                                          size_t p0, int gt, uint8_t *stage_a, uint8_t *stage_b) {
  for (int it = gt; it < TL * (TM / 4); it += GT) {
    const int l = it / (TM / 4), q = it - l * (TM / 4);
    const size_t p = p0 + 4 * q;
    const size_t i = base + (size_t)l * N + p;
    uint8_t *da = stage_a + (size_t)(l * TM + 4 * q) * 4, *db = stage_b + (size_t)(l * TM + 4 * q) * 4;
    if (p + 4 <= N) {
      cp16(da, xt + i);
      cp16(db, x + i);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        reinterpret_cast<float *>(da)[e] = p + e < N ? xt[i + e] : 0.f;
        reinterpret_cast<float *>(db)[e] = p + e < N ? x[i + e] : 0.f;
      }
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// the band rows stage_raw will read for (base, p0), into L2 ahead of time:
// one bulk prefetch per (band, array), 16-byte aligned (p0 is a multiple of
// the 128-pixel tile) and cut at the end of the pixel range
__device__ __forceinline__ void prefetch_raw(const float *xt, const float *x, size_t base,
                                             size_t N, size_t p0, int gt) {
  if (gt >= 2 * TL || p0 >= N) return;
  const size_t cnt = (N - p0 < (size_t)TM ? N - p0 : (size_t)TM) & ~(size_t)3;
  if (cnt == 0) return;
  const int l = gt >> 1;
  const float *src = (gt & 1 ? x : xt) + base + (size_t)l * N + p0;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"((uint32_t)(cnt * 4))
               : "memory");
}

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(GT) : "memory");
}

// 3 x 8 MMAs of one TF32-split product into tensor-memory columns d; with
// acc the product is added to what d holds
__device__ __forceinline__ void issue_product(uint32_t d, uint32_t ahi, uint32_t alo,
                                              uint32_t bhi, uint32_t blo, bool acc) {
#pragma unroll 1
  for (int ks = 0; ks < TL / 8; ++ks) {
    const uint32_t ko = (uint32_t)ks * 256u;   // two core matrices along K
    const uint64_t dah = sdesc(ahi + ko), dal = sdesc(alo + ko);
    const uint64_t dbh = sdesc(bhi + ko), dbl = sdesc(blo + ko);
    const uint32_t first = ks == 0 && !acc;
    asm volatile("{\n\t.reg .pred p;\n\tsetp.eq.u32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d), "l"(dal), "l"(dbh), "r"(IDESC), "r"(first) : "memory");
    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                 ::"r"(d), "l"(dah), "l"(dbl), "r"(IDESC) : "memory");
    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                 ::"r"(d), "l"(dah), "l"(dbh), "r"(IDESC) : "memory");
  }
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(mbar) : "memory");
}

// bounded wait for the phase `ph` of an mbarrier; true when it completed
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t ph, long spin) {
  uint32_t done = 0;
  for (long it = 0; it < spin && !done; ++it)
    asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}" : "=r"(done) : "r"(mbar), "r"(ph) : "memory");
  return done != 0;
}

// the thread's 32 accumulator columns [c0, c0 + 32) of its lane
__device__ __forceinline__ void tmem_row32(uint32_t taddr, float (&o)[32]) {
  uint32_t v[32];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(v[16 * h + 0]), "=r"(v[16 * h + 1]), "=r"(v[16 * h + 2]), "=r"(v[16 * h + 3]),
                   "=r"(v[16 * h + 4]), "=r"(v[16 * h + 5]), "=r"(v[16 * h + 6]), "=r"(v[16 * h + 7]),
                   "=r"(v[16 * h + 8]), "=r"(v[16 * h + 9]), "=r"(v[16 * h + 10]), "=r"(v[16 * h + 11]),
                   "=r"(v[16 * h + 12]), "=r"(v[16 * h + 13]), "=r"(v[16 * h + 14]), "=r"(v[16 * h + 15])
                 : "r"(taddr + 16u * h) : "memory");
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) o[j] = __uint_as_float(v[j]);
}

// the thread's 32 values as TF32 halves into row `row`, columns [32h, 32h+32)
__device__ __forceinline__ void store_split(uint8_t *ahi, uint8_t *alo, int row, int h,
                                            const float (&z)[32]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float hi[4], lo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      hi[e] = tf32r(z[4 * q + e]);
      lo[e] = tf32r(z[4 * q + e] - hi[e]);
    }
    const uint32_t o = cm_off(row, 32 * h + 4 * q);
    *reinterpret_cast<float4 *>(ahi + o) = make_float4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<float4 *>(alo + o) = make_float4(lo[0], lo[1], lo[2], lo[3]);
  }
}

template <int CH>
__global__ void __launch_bounds__(CTA_T, 1) k_dct_tc(TcArgs a) {
  extern __shared__ uint8_t raw[];
  __shared__ __align__(8) uint64_t mbar[NG];
  __shared__ uint32_t tmem_base;
  __shared__ int bail[NG];
  uint8_t *base = reinterpret_cast<uint8_t *>(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  uint8_t *cth[4] = {base, base + CMAT_B, base + 2 * CMAT_B, base + 3 * CMAT_B};  // Chi Clo CThi CTlo
  const int tid = threadIdx.x, g = tid / GT, gt = tid % GT, wg = gt >> 5, lane = tid & 31;
  uint8_t *ahi = base + 4 * CMAT_B + (size_t)g * 2 * TILE_B, *alo = ahi + TILE_B;
  // C tables into the operand layout: row = output index, column = summed index
  const float *src[4] = {a.chi, a.clo, a.cthi, a.ctlo};
#pragma unroll
  for (int m = 0; m < 4; ++m)
    for (int i = tid; i < TL * TL; i += CTA_T)
      *reinterpret_cast<float *>(cth[m] + cm_off(i / TL, i % TL)) = src[m][i];
  if (tid < NG) {
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar[tid]);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    bail[tid] = 0;
  }
  if (tid < 32) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(dst), "r"(tmem_cols(CH)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar[g]);
  const uint32_t quad = (uint32_t)(wg & 3), h = (uint32_t)(wg >> 2);
  // accumulators of the group: [0, 64) first product of chains 0 and 2,
  // [64, 128) second product of chains 0 and 2 (one chain: nothing else);
  // three chains add [128, 192), [192, 256) for chain 1.  Chain 2 (d/dgamma)
  // multiplies gamma z'_gamma + z and gamma v'_gamma + v (Algorithm 4): its
  // products are accumulated onto chain 0's, C (gamma z') + C z, so chain
  // 0's tiles are neither staged nor reloaded again.
  const uint32_t lanes = tmem_base + ((quad * 32u) << 16) + (uint32_t)g * group_cols(CH);
  const uint32_t gcol = tmem_base + (uint32_t)g * group_cols(CH);   // MMA destinations
  const uint32_t sa_hi = (uint32_t)__cvta_generic_to_shared(ahi);
  const uint32_t sa_lo = (uint32_t)__cvta_generic_to_shared(alo);
  const uint32_t sc_hi = (uint32_t)__cvta_generic_to_shared(cth[0]);
  const uint32_t sc_lo = (uint32_t)__cvta_generic_to_shared(cth[1]);
  const uint32_t sct_hi = (uint32_t)__cvta_generic_to_shared(cth[2]);
  const uint32_t sct_lo = (uint32_t)__cvta_generic_to_shared(cth[3]);
  const size_t N = a.npix;
  const size_t CS = (size_t)a.B * TL * N;
  const int tpc = (int)((N + TM - 1) / TM);
  const int ntiles = tpc * a.B;
  const int row = (int)quad * 32 + lane;          // pixel within the tile = accumulator lane
  uint32_t ph = 0;
  bool ok = true;

  for (int tile = blockIdx.x * NG + g; tile < ntiles && ok; tile += gridDim.x * NG) {
    const int cube = tile / tpc;
    const size_t p = (size_t)(tile - cube * tpc) * TM + row;
    const bool valid = p < N;
    const float gamma = (float)a.sc[cube].gamma, sigma = (float)a.sc[cube].sigma;
    const float al = valid ? a.alpha[(size_t)cube * N + p] : 0.f;
    const size_t pix = (size_t)cube * TL * N + p + (size_t)(32 * h) * N;   // band 32h of the cube
    uint32_t keep = 0;
#pragma unroll 1
    for (int c = 0; c < CH && ok; ++c) {
      const bool mix = CH == 3 && c == 2;          // accumulate onto chain 0's products
      const uint32_t off1 = (CH == 3 && c == 1) ? 128u : 0u, off2 = off1 + 64u;
      // ---- first product: z = 2x~ - x (gamma z' for d/dgamma, whose + z is
      // chain 0's product already in tensor memory); the raw tiles are staged
      // through the A buffers, free at this point
      const size_t tile_base = (size_t)cube * TL * N;
      const size_t p0 = p - row;
      float z[32];
      stage_raw(a.xt + c * CS, a.x + c * CS, tile_base, N, p0, gt, ahi, alo);
      {   // the next (tile, chain) of this group, into L2 while this one runs
        const int nt = c + 1 < CH ? tile : tile + (int)gridDim.x * NG;
        const int nc = c + 1 < CH ? c + 1 : 0;
        if (nt < ntiles) {
          const int ncube = nt / tpc;
          prefetch_raw(a.xt + nc * CS, a.x + nc * CS, (size_t)ncube * TL * N, N,
                       (size_t)(nt - ncube * tpc) * TM, gt);
        }
      }
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      group_sync(g);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int o = ((32 * (int)h + j) * TM + row) * 4;
        z[j] = 2.f * *reinterpret_cast<const float *>(ahi + o) -
               *reinterpret_cast<const float *>(alo + o);
      }
      if (mix) {
#pragma unroll
        for (int j = 0; j < 32; ++j) z[j] *= gamma;
      }
      group_sync(g);                       // staging reads done before the split overwrites it
      store_split(ahi, alo, row, (int)h, z);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      group_sync(g);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (gt == 0 && !a.inject) {
        issue_product(gcol + off1, sa_hi, sa_lo, sc_hi, sc_lo, mix);
        commit(mb);
      }
      // old duals while the product runs
      float vo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) vo[j] = valid ? a.v[c * CS + pix + (size_t)j * N] : 0.f;
      if (!wait_phase(mb, ph, a.spin)) bail[g] = 1;
      ph ^= 1u;
      group_sync(g);
      if (bail[g]) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float acc[32];
      tmem_row32(lanes + off1 + 32u * h, acc);
      // ---- dual update (chain 0 sets the masks Pi(v~) used by the others)
      const float sg = (c == 2 ? sigma : sigma * gamma) * al;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float vt = fmaf(sg, acc[j], vo[j]);
        float vn;
        if (c == 0) {
          vn = satf(vt);
          if (fabsf(vt) <= 1.f) keep |= 1u << j;
        } else {
          vn = (keep >> j) & 1u ? vt : 0.f;
        }
        if (!valid) vn = 0.f;
        else a.v[c * CS + pix + (size_t)j * N] = vn;
        z[j] = vn;
      }
      if (mix) {                           // gamma v'_gamma (+ v: chain 0's product)
#pragma unroll
        for (int j = 0; j < 32; ++j) z[j] *= gamma;
      }
      // ---- second product: t = gamma_n C^T v
      store_split(ahi, alo, row, (int)h, z);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      group_sync(g);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (gt == 0 && !a.inject) {
        issue_product(gcol + off2, sa_hi, sa_lo, sct_hi, sct_lo, mix);
        commit(mb);
      }
      if (!wait_phase(mb, ph, a.spin)) bail[g] = 1;
      ph ^= 1u;
      group_sync(g);
      if (bail[g]) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      tmem_row32(lanes + off2 + 32u * h, acc);
      const float s2 = (c == 2) ? al : gamma * al;
      if (valid) {
#pragma unroll
        for (int j = 0; j < 32; ++j) a.t[c * CS + pix + (size_t)j * N] = s2 * acc[j];
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
  }
  if (!ok) {
    if (gt == 0) atomicExch(a.err, 1);
    wait_phase(mb, ph, a.spin);  // let an MMA still in flight finish before freeing
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 ::"r"(tmem_base), "r"(tmem_cols(CH)) : "memory");
}

template <int CH>
cudaError_t launch_tc(const TcArgs &a, cudaStream_t st, Prof *prof) {
  static bool attr = false;
  static int sms = 0;
  if (!attr) {
    cudaFuncSetAttribute(k_dct_tc<CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    attr = true;
  }
  const size_t N = a.npix;
  const size_t ntiles = ((N + TM - 1) / TM) * (size_t)a.B;
  const size_t ctas = (ntiles + NG - 1) / NG;
  const size_t grid = ctas < (size_t)sms ? ctas : (size_t)sms;
  const double vox = (double)N * TL * a.B;
  ProfScope ps(prof, "spectral_dual", CH * vox * 20.0, 2.0 * CH * 2.0 * TL * vox, st);
  k_dct_tc<CH><<<(unsigned)grid, CTA_T, SMEM, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t dct_dual_tc(const DctArgs &d, const Group &gr, int *err, cudaStream_t st) {
  if (d.L != TL || d.Lp != TL) return cudaErrorInvalidValue;
  TcArgs a{};
  a.n = d.n; a.L = d.L; a.B = d.B > 0 ? d.B : 1;
  a.npix = d.npix ? d.npix : (size_t)d.n * d.n;
  a.chi = d.chi; a.clo = d.clo; a.cthi = d.cthi; a.ctlo = d.ctlo;
  a.alpha = d.alpha; a.sc = d.sc;
  a.xt = gr.xt; a.x = gr.x; a.v = gr.v; a.t = gr.t; a.err = err;
  a.inject = d.inject_timeout;
  a.spin = d.inject_timeout ? kSpinInjected : kSpin;
  if (gr.C == 3) return launch_tc<3>(a, st, d.prof);
  return launch_tc<1>(a, st, d.prof);
}

}  // namespace muffin
