// Per-band noise level of a dirty cube by the median absolute deviation
// (Sec. 3.1 names MAD-type robust statistics as the way to estimate the
// noise variances in the image domain).  Reading: the finest diagonal
// (high-high) band of the orthonormal Haar transform of each dirty image,
//   d[i][j] = (y[2i][2j] - y[2i][2j+1] - y[2i+1][2j] + y[2i+1][2j+1]) / 2,
// sigma_l = median(|d - median(d)|) / Phi^-1(3/4); the median of an even
// count is the mean of the two middle values.
//
// Medians are exact order statistics found by radix selection: float values
// map to order-preserving 32-bit keys, and four passes of an 8-bit
// histogram (one CTA per band, shared-memory atomics) narrow the key down
// to the k-th smallest.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace muffin {

namespace {

constexpr int kSelThreads = 1024;
constexpr double kPhiInv34 = 0.6744897501960817;   // Phi^-1(3/4)

__device__ __forceinline__ uint32_t fkey(float v) {
  const uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float kfloat(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// d[l][i][j]: the finest high-high Haar coefficients of every band
__global__ void k_haar_hh(const float *__restrict__ y, float *__restrict__ d, int n, int L) {
  const int h = n >> 1;
  const size_t per = (size_t)h * h, total = per * L;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t l = t / per, r = t - l * per;
    const int i = (int)(r / h), j = (int)(r - (size_t)i * h);
    const float *p = y + l * (size_t)n * n + (size_t)(2 * i) * n + 2 * j;
    const float a = p[0], b = p[1], c = p[n], e = p[n + 1];
    d[t] = 0.5f * ((a - b) - (c - e));
  }
}

// the k-th smallest key (0-based) of band blockIdx.x's M values v(i), where
// v(i) = d[i] (center == NULL) or |d[i] - center[band]| rounded to float
__device__ uint32_t select_key(const float *__restrict__ d, size_t M, const double *center,
                               long long k, uint32_t *hist, uint32_t *shared_state) {
  uint32_t prefix = 0, mask = 0;
  const double c = center ? center[blockIdx.x] : 0.0;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (size_t i = threadIdx.x; i < M; i += blockDim.x) {
      const float v = center ? (float)fabs((double)d[i] - c) : d[i];
      const uint32_t key = fkey(v);
      if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long cum = 0;
      int b = 0;
      for (; b < 255; ++b) {
        if (cum + (long long)hist[b] > k) break;
        cum += hist[b];
      }
      shared_state[0] = (uint32_t)b;
      shared_state[1] = (uint32_t)(k - cum);
    }
    __syncthreads();
    prefix |= shared_state[0] << shift;
    mask |= 0xffu << shift;
    k = shared_state[1];
    __syncthreads();
  }
  return prefix;
}

// one CTA per band: the median of d (center == NULL) or of |d - center|
__global__ void __launch_bounds__(kSelThreads)
k_median(const float *__restrict__ d, size_t M, const double *center, double *out) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t st[2];
  const float *db = d + (size_t)blockIdx.x * M;
  const uint32_t lo = select_key(db, M, center, (long long)((M - 1) / 2), hist, st);
  const uint32_t hi = (M & 1) ? lo : select_key(db, M, center, (long long)(M / 2), hist, st);
  if (threadIdx.x == 0) out[blockIdx.x] = 0.5 * ((double)kfloat(lo) + (double)kfloat(hi));
}

__global__ void k_mad_var(const double *mad, double *var, int L) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < L) {
    const double s = mad[l] / kPhiInv34;
    var[l] = s * s;
  }
}

}  // namespace

cudaError_t noise_mad(const float *y, int n, int L, float *d_scratch, double *med,
                      double *mad, double *var, cudaStream_t st) {
  const size_t M = (size_t)(n / 2) * (n / 2);
  const size_t total = M * L;
  const int nb = (int)((total + 255) / 256 > 152 * 16 ? 152 * 16 : (total + 255) / 256);
  k_haar_hh<<<nb > 0 ? nb : 1, 256, 0, st>>>(y, d_scratch, n, L);
  k_median<<<L, kSelThreads, 0, st>>>(d_scratch, M, nullptr, med);
  k_median<<<L, kSelThreads, 0, st>>>(d_scratch, M, med, mad);
  k_mad_var<<<(L + 127) / 128, 128, 0, st>>>(mad, var, L);
  return cudaGetLastError();
}

}  // namespace muffin
