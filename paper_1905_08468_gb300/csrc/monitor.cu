// FP64 reductions of the convergence monitor (Sec. 2.1: the iteration has
// no closed form, so it is run until its iterates settle):
//   * per band, sum (x - x_prev)^2, sum x_prev^2 and the number of NaN/Inf
//     entries of x (the relative change ||X^k - X^{k-1}|| / ||X^{k-1}|| and
//     the numeric-failure scan share one pass);
//   * per band, sum (scale w - y)^2 over an FP64 image w (the data term of
//     Eq. probopt, from an FP64 forward convolution H x);
//   * per band, sum a_i |u_i| (the l1 terms of Eq. RegAll, with the pixel
//     weights alpha_n for the spectral term).
// Every reduction is two-pass and in a fixed order (deterministic).
#include <cuda_runtime.h>

#include "kernels.h"

namespace muffin {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBpb = 16;   // blocks per band

template <int NV>
__device__ void block_sum_nv(double (&v)[NV], double *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[wid * NV + q] = v[q];
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = lane < nw ? sh[lane * NV + q] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      v[q] = s;
    }
  }
  __syncthreads();
}

// grid (bpb, L); part[(l * bpb + blk) * 3 + q]
__global__ void k_mon_state(const float *__restrict__ x, const float *__restrict__ xo,
                            size_t N, double *__restrict__ part) {
  const size_t base = (size_t)blockIdx.y * N;
  double v[3] = {0.0, 0.0, 0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    const float a = x[base + i];
    if (!isfinite(a)) v[2] += 1.0;
    if (xo) {
      const double p = xo[base + i], d = (double)a - p;
      v[0] = fma(d, d, v[0]);
      v[1] = fma(p, p, v[1]);
    } else {
      v[1] = fma((double)a, (double)a, v[1]);
    }
  }
  __shared__ double sh[32 * 3];
  block_sum_nv<3>(v, sh);
  if (threadIdx.x == 0) {
    double *p = part + 3 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
    p[0] = v[0]; p[1] = v[1]; p[2] = v[2];
  }
}

__global__ void k_mon_resid(const double2 *__restrict__ w, const float *__restrict__ y,
                            double scale, size_t N, double *__restrict__ part) {
  const size_t base = (size_t)blockIdx.y * N;
  double v[1] = {0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    const double r = scale * w[base + i].x - (double)y[base + i];
    v[0] = fma(r, r, v[0]);
  }
  __shared__ double sh[32];
  block_sum_nv<1>(v, sh);
  if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = v[0];
}

// weights alpha[(l / Lc) * N + (i mod N)] when alpha != NULL
__global__ void k_mon_abs(const float *__restrict__ u, size_t per_band,
                          const float *__restrict__ alpha, int Lc, size_t N,
                          double *__restrict__ part) {
  const int l = blockIdx.y;
  const size_t base = (size_t)l * per_band;
  const float *al = alpha ? alpha + (size_t)(l / Lc) * N : nullptr;
  double v[1] = {0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < per_band;
       i += (size_t)gridDim.x * blockDim.x) {
    const double a = fabs((double)u[base + i]);
    v[0] += al ? a * (double)al[i % N] : a;
  }
  __shared__ double sh[32];
  block_sum_nv<1>(v, sh);
  if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = v[0];
}

// out[l * nv + q] = sum over the band's bpb partials, fixed order
__global__ void k_mon_final(const double *__restrict__ part, int nv, int bpb,
                            double *__restrict__ out) {
  if (threadIdx.x >= (unsigned)nv) return;
  const int l = blockIdx.x;
  double s = 0.0;
  for (int b = 0; b < bpb; ++b) s += part[((size_t)l * bpb + b) * nv + threadIdx.x];
  out[(size_t)l * nv + threadIdx.x] = s;
}

__global__ void k_mul_c64(double2 *__restrict__ a, const double2 *__restrict__ h,
                          size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    const double2 p = a[i], q = h[i];
    a[i] = make_double2(p.x * q.x - p.y * q.y, p.x * q.y + p.y * q.x);
  }
}

__global__ void k_twice_minus(const float *__restrict__ xt, const float *__restrict__ x,
                              float *__restrict__ z, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    z[i] = 2.f * xt[i] - x[i];
}

int bpb_for(size_t per_band) {
  const size_t g = (per_band + kThreads - 1) / kThreads;
  return (int)(g > kMaxBpb ? kMaxBpb : (g ? g : 1));
}

}  // namespace

size_t monitor_scratch_doubles(int L) { return (size_t)L * (3 * kMaxBpb + 12) + 64; }

cudaError_t mon_state(const float *x, const float *xo, int L, size_t N, double *scratch,
                      double *out, cudaStream_t st) {
  const int bpb = bpb_for(N);
  k_mon_state<<<dim3(bpb, L), kThreads, 0, st>>>(x, xo, N, scratch);
  k_mon_final<<<L, 32, 0, st>>>(scratch, 3, bpb, out);
  return cudaGetLastError();
}

cudaError_t mon_resid2(const double2 *w, const float *y, double scale, int L, size_t N,
                       double *scratch, double *out, cudaStream_t st) {
  const int bpb = bpb_for(N);
  k_mon_resid<<<dim3(bpb, L), kThreads, 0, st>>>(w, y, scale, N, scratch);
  k_mon_final<<<L, 32, 0, st>>>(scratch, 1, bpb, out);
  return cudaGetLastError();
}

cudaError_t mon_abs(const float *u, int L, size_t per_band, const float *alpha, int Lc,
                    size_t N, double *scratch, double *out, cudaStream_t st) {
  const int bpb = bpb_for(per_band);
  k_mon_abs<<<dim3(bpb, L), kThreads, 0, st>>>(u, per_band, alpha, Lc, N, scratch);
  k_mon_final<<<L, 32, 0, st>>>(scratch, 1, bpb, out);
  return cudaGetLastError();
}

cudaError_t twice_minus(const float *xt, const float *x, float *z, size_t count,
                        cudaStream_t st) {
  const size_t g = (count + 255) / 256;
  const int nb = (int)(g > 152 * 16 ? 152 * 16 : (g ? g : 1));
  k_twice_minus<<<nb, 256, 0, st>>>(xt, x, z, count);
  return cudaGetLastError();
}

cudaError_t mul_c64(double2 *a, const double2 *h, size_t count, cudaStream_t st) {
  const size_t g = (count + 255) / 256;
  const int nb = (int)(g > 152 * 16 ? 152 * 16 : (g ? g : 1));
  k_mul_c64<<<nb, 256, 0, st>>>(a, h, count);
  return cudaGetLastError();
}

}  // namespace muffin
