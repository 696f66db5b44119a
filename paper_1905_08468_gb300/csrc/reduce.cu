// FP64 reductions: Lipschitz constant, per-band energies and the ADA-PT
// statistics (Eqs. SUGAR, PSURE0) with the theta update of Eq. (adaptgrad).
//
// All reductions are deterministic: each block writes its partial sums and
// one block combines them in a fixed order, so a resumed run reproduces an
// uninterrupted one bit for bit.
#include <cuda_runtime.h>

#include "kernels.h"

namespace muffin {

namespace {

constexpr int kRedThreads = 256;
constexpr int kMaxBlocks = 1024;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// block-wide sum of NV doubles held by every thread; result valid in thread 0
template <int NV>
__device__ void block_sum(double (&v)[NV], double *sh /* [32][NV] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[wid * NV + q] = v[q];
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = lane < nw ? sh[lane * NV + q] : 0.0;
      v[q] = warp_sum(s);
    }
  }
  __syncthreads();
}

__global__ void k_max_abs2(const double2 *__restrict__ h, size_t count,
                           double *__restrict__ part) {
  double m = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    const double2 z = h[i];
    m = fmax(m, z.x * z.x + z.y * z.y);
  }
  __shared__ double sh[32];
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    m = warp_max(m);
    if (threadIdx.x == 0) part[blockIdx.x] = m;
  }
}

__global__ void k_max_final(const double *__restrict__ part, int nb,
                            double *__restrict__ out) {
  double m = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) m = fmax(m, part[i]);
  __shared__ double sh[32];
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    m = warp_max(m);
    if (threadIdx.x == 0) *out = m;
  }
}

// grid (blocks_per_band, L); partials [L][blocks_per_band]
__global__ void k_band_sumsq(const float *__restrict__ y, size_t per_band,
                             double *__restrict__ part) {
  const float *yb = y + (size_t)blockIdx.y * per_band;
  double v[1] = {0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < per_band;
       i += (size_t)gridDim.x * blockDim.x) {
    const double t = yb[i];
    v[0] += t * t;
  }
  __shared__ double sh[32];
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = v[0];
}

__global__ void k_band_final(const double *__restrict__ part, int nb,
                             double *__restrict__ out) {
  double v[1] = {0.0};
  // fixed order: thread i sums i, i+bs, ...; then the tree
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v[0] += part[blockIdx.x * nb + i];
  __shared__ double sh[32];
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = v[0];
}

__global__ void k_axpy(const float *__restrict__ y, const float *__restrict__ d,
                       float eps, float *__restrict__ out, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = y[i] + eps * d[i];
}

// grid (blocks_per_band, L).  Four pixels per step: the six products of
// each pixel in FP32 (the differences of the two groups' FP32 iterates are
// exact when they are close), the four pixels' sums in FP32, then every
// further sum in FP64 in a fixed order (deterministic).
__global__ void k_sure_stats(SureStatsArgs a, double *__restrict__ part) {
  const size_t N = (size_t)a.n * a.n;
  const size_t CL = (size_t)a.L * N;   // stride between chains of a group
  const int l = blockIdx.y;
  const double w = a.wband[l];
  const size_t base = (size_t)l * N;
  double v[6] = {0, 0, 0, 0, 0, 0};
  const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  if ((N & 3) == 0) {
    const float4 *gr4 = reinterpret_cast<const float4 *>(a.grad + base);
    const float4 *hd4 = reinterpret_cast<const float4 *>(a.htd + base);
    const float4 *b4 = reinterpret_cast<const float4 *>(a.b + base);
    const float4 *x04 = reinterpret_cast<const float4 *>(a.x + base);
    const float4 *xm4 = reinterpret_cast<const float4 *>(a.x + CL + base);
    const float4 *xg4 = reinterpret_cast<const float4 *>(a.x + 2 * CL + base);
    const float4 *y04 = reinterpret_cast<const float4 *>(a.xb + base);
    const float4 *ym4 = reinterpret_cast<const float4 *>(a.xb + CL + base);
    const float4 *yg4 = reinterpret_cast<const float4 *>(a.xb + 2 * CL + base);
    for (size_t q = t0; q < (N >> 2); q += stride) {
      const float4 gr = gr4[q], hd = hd4[q], bb = b4[q];
      const float4 x0 = x04[q], xm = xm4[q], xg = xg4[q];
      const float4 y0 = y04[q], ym = ym4[q], yg = yg4[q];
      float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      auto one = [&](float g, float h, float b, float p0, float pm, float pg, float q0,
                     float qm, float qg) {
        s[0] = fmaf(g, pm, s[0]);
        s[1] = fmaf(g, pg, s[1]);
        s[2] = fmaf(qm - pm, h, s[2]);
        s[3] = fmaf(qg - pg, h, s[3]);
        s[4] = fmaf(p0, g - b, s[4]);
        s[5] = fmaf(q0 - p0, h, s[5]);
      };
      one(gr.x, hd.x, bb.x, x0.x, xm.x, xg.x, y0.x, ym.x, yg.x);
      one(gr.y, hd.y, bb.y, x0.y, xm.y, xg.y, y0.y, ym.y, yg.y);
      one(gr.z, hd.z, bb.z, x0.z, xm.z, xg.z, y0.z, ym.z, yg.z);
      one(gr.w, hd.w, bb.w, x0.w, xm.w, xg.w, y0.w, ym.w, yg.w);
#pragma unroll
      for (int k = 0; k < 6; ++k) v[k] += (double)s[k];
    }
  } else {
    for (size_t i = t0; i < N; i += stride) {
      const size_t j = base + i;
      const double gr = a.grad[j];
      const double hd = a.htd[j];
      const double xm = a.x[CL + j], xg = a.x[2 * CL + j];
      const double xbm = a.xb[CL + j], xbg = a.xb[2 * CL + j];
      const double x0 = a.x[j], xb0 = a.xb[j];
      v[0] += gr * xm;
      v[1] += gr * xg;
      v[2] += (xbm - xm) * hd;
      v[3] += (xbg - xg) * hd;
      v[4] += x0 * (gr - (double)a.b[j]);
      v[5] += (xb0 - x0) * hd;
    }
  }
  v[2] *= w; v[3] *= w; v[5] *= w;
  __shared__ double sh[32 * 6];
  block_sum<6>(v, sh);
  if (threadIdx.x == 0) {
    double *p = part + 6 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
    for (int q = 0; q < 6; ++q) p[q] = v[q];
  }
}

// one block per cube: cube b's partials are bands [b L, (b+1) L) x bpb
__global__ void k_theta_update(ThetaUpdateArgs a) {
  const int b = blockIdx.x;
  const double *part = a.partials + (size_t)b * a.nb_per_cube * 6;
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < a.nb_per_cube; i += blockDim.x)
    for (int q = 0; q < 6; ++q) v[q] += part[6 * (size_t)i + q];
  __shared__ double sh[32 * 6];
  block_sum<6>(v, sh);
  if (threadIdx.x == 0) {
    DevScalars *sc = a.sc + b;
    const double *cc = a.cube_const + 4 * b;   // psure_const, lipschitz, Bsum, Asum
    double *rec = a.record + ((size_t)(*a.rec_count) * a.B + b) * 7;
    const double mu = sc->mu, gamma = sc->gamma;
    const double sug_mu = 2.0 * v[0] + v[2];
    const double sug_ga = 2.0 * v[1] + v[3];
    const double psure = cc[0] + v[4] + v[5];
    rec[0] = 0.0;
    rec[1] = mu;
    rec[2] = gamma;
    rec[3] = sug_mu;
    rec[4] = sug_ga;
    rec[5] = psure;
    rec[6] = sc->tau;
    // explicit fused products: the host-side descent (muffin_sure_global_auto)
    // applies the same rounding
    const double nmu = fmax(fma(-a.eta_mu, sug_mu, mu), a.theta_min);
    const double nga = fmax(fma(-a.eta_gamma, sug_ga, gamma), a.theta_min);
    sc->mu = nmu;
    sc->gamma = nga;
    sc->tau = a.tau_fixed > 0
                  ? a.tau_fixed
                  : a.safety / (0.5 * cc[1] + sc->sigma * (a.K * nmu * nmu * cc[2] + nga * nga * cc[3]));
  }
}

__global__ void k_bump(int *counter) { *counter += 1; }

}  // namespace

cudaError_t max_abs2_c64(const double2 *hh, size_t count, double *scratch,
                         double *out, cudaStream_t st) {
  size_t g = (count + kRedThreads - 1) / kRedThreads;
  const int nb = (int)(g > kMaxBlocks ? kMaxBlocks : (g ? g : 1));
  k_max_abs2<<<nb, kRedThreads, 0, st>>>(hh, count, scratch);
  k_max_final<<<1, kRedThreads, 0, st>>>(scratch, nb, out);
  return cudaGetLastError();
}

cudaError_t band_sumsq(const float *y, int L, size_t per_band, double *out,
                       cudaStream_t st) {
  // out must have room for L + L*bpb doubles; partials placed after the L results
  size_t g = (per_band + kRedThreads - 1) / kRedThreads;
  const int bpb = (int)(g > 64 ? 64 : (g ? g : 1));
  double *part = out + L;
  k_band_sumsq<<<dim3(bpb, L), kRedThreads, 0, st>>>(y, per_band, part);
  k_band_final<<<L, kRedThreads, 0, st>>>(part, bpb, out);
  return cudaGetLastError();
}

// alpha[b][n] = 1 / (sqrt(sum_l x[b][l][n]^2) + eps): the norm of pixel
// n's spectrum, which equals ||W_lambda x^n||_2 for the orthonormal DCT
// (Eq. 2regpar weights); FP64 sum in band order
__global__ void k_pixel_weights(const float *__restrict__ x, int B, int L, size_t N,
                                double eps, float *__restrict__ alpha) {
  const size_t total = (size_t)B * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / N, px = i - b * N;
    const float *xb = x + b * L * N + px;
    double s = 0.0;
    for (int l = 0; l < L; ++l) {
      const double v = xb[(size_t)l * N];
      s = fma(v, v, s);
    }
    alpha[i] = (float)(1.0 / (sqrt(s) + eps));
  }
}

cudaError_t pixel_weights(const float *x, int B, int L, size_t N, double eps, float *alpha,
                          cudaStream_t st) {
  const size_t g = ((size_t)B * N + 255) / 256;
  const int nb = (int)(g > 152 * 16 ? 152 * 16 : (g ? g : 1));
  k_pixel_weights<<<nb, 256, 0, st>>>(x, B, L, N, eps, alpha);
  return cudaGetLastError();
}

cudaError_t axpy_f32(const float *y, const float *d, float eps, float *out,
                     size_t count, cudaStream_t st) {
  size_t g = (count + 255) / 256;
  const int nb = (int)(g > 152 * 32 ? 152 * 32 : (g ? g : 1));
  k_axpy<<<nb, 256, 0, st>>>(y, d, eps, out, count);
  return cudaGetLastError();
}

cudaError_t sure_stats(const SureStatsArgs &a, double *partials, int *nblocks,
                       cudaStream_t st) {
  const size_t N = (size_t)a.n * a.n;
  size_t g = (N + kRedThreads - 1) / kRedThreads;
  int bpb = (int)(g > 16 ? 16 : (g ? g : 1));
  // keep total partial count bounded: L * bpb <= 4096
  while (bpb > 1 && (size_t)a.L * bpb > 4096) bpb >>= 1;
  k_sure_stats<<<dim3(bpb, a.L), kRedThreads, 0, st>>>(a, partials);
  *nblocks = bpb;
  return cudaGetLastError();
}

cudaError_t theta_update(const ThetaUpdateArgs &a, cudaStream_t st) {
  k_theta_update<<<a.B, kRedThreads, 0, st>>>(a);
  k_bump<<<1, 1, 0, st>>>(a.rec_count);
  return cudaGetLastError();
}

}  // namespace muffin
