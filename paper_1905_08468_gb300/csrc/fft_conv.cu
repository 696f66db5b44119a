// Least-squares gradient H_l^T (H_l x_l - y_l) of Algorithm 2 (eq. grad2)
// and H_l^T H_l x'_l of Algorithms 3/4, by 2D FFT (Eq. model read as a
// circular convolution).  Since H_l^T H_l = F^-1 diag(|h_hat_l|^2) F and
// b_l = H_l^T y_l is fixed per call, the hot path computes
//     g = F^-1 ( |h_hat|^2 . F x ) - b
// in three FP32 passes over the cube:
//   1. rows:    pairs of real rows packed as one complex row, FFT, split into
//               the two half spectra (n/2+1 bins), stored kx-major ("columns
//               contiguous") so that pass 2 reads whole columns;
//   2. columns: forward FFT of each column, multiply by |h_hat|^2 / n^2,
//               inverse FFT, in place;
//   3. rows:    rebuild the Hermitian row spectra of two rows at a time,
//               inverse FFT, subtract b, store.
// The FP64 2D transform at the bottom is used only when a plan or call is
// set up (PSF spectra, H^T y, H^T delta).
#include <cuda_runtime.h>

#include "fft.cuh"
#include "fft32.cuh"
#include "kernels.h"

namespace muffin {

namespace {

constexpr int kThreads = 256;

// sequences per CTA so that every thread owns fft_vpt(n) values per stage
__host__ __device__ constexpr int seqs_per_cta(int n) { return kThreads * fft_vpt(n) / n; }
// complex (row-pair) sequences per CTA of the row passes: 2 * nq real rows
__host__ __device__ constexpr int row_pairs(int n) { return seqs_per_cta(n) < n / 2 ? seqs_per_cta(n) : n / 2; }

// stage the twiddle tables (tlen entries) into shared memory
__device__ __forceinline__ void load_tw(float2 *dst, const float2 *__restrict__ src, int tlen) {
  for (int i = threadIdx.x; i < tlen; i += blockDim.x) dst[i] = src[i];
}

template <int NN, int RMAX>
__global__ void __launch_bounds__(kThreads)
k_rows_fwd(const float *__restrict__ x, float2 *__restrict__ S,
           const float2 *__restrict__ tw, int tlen, int img0) {
  // sizes are compile-time so that the index splits below are shifts
  constexpr int n = NN, nq = row_pairs(NN), nh = (NN >> 1) + 1;
  constexpr int pitch = n + (n >> 4);
  extern __shared__ float2 sm2[];
  const int img = blockIdx.y;           // image of the chunk (its spectrum in S)
  const int gimg = img0 + img;          // image of the cube
  const int y0 = blockIdx.x * 2 * nq;
  float2 *d = sm2, *tws = sm2 + nq * pitch;
  load_tw(tws, tw, tlen);
  // element u of the thread is i = tid + 256 u of the [nq][n] row pairs:
  // pair tid / n + 256 u / n, column tid % n + (256 u) % n, so every index
  // is a per-thread base plus a compile-time offset
  const int tid = threadIdx.x;
  const float *xi = x + (size_t)gimg * n * n + (size_t)(y0 + 2 * (tid / n)) * n + tid % n;
  const int sb = (tid / n) * pitch + fpad(tid % n);
  constexpr int VPT = fft_vpt(NN);
  float2 v[VPT];
#pragma unroll
  for (int u = 0; u < VPT; ++u) {
    const int q = (kThreads * u) / n, c = (kThreads * u) % n;
    if (tid + u * kThreads < nq * n)
      v[u] = make_float2(xi[2 * q * n + c], xi[(2 * q + 1) * n + c]);
  }
#pragma unroll
  for (int u = 0; u < VPT; ++u) {
    const int q = (kThreads * u) / n, c = (kThreads * u) % n;
    if (tid + u * kThreads < nq * n) d[sb + q * pitch + fpad(c)] = v[u];
  }
  __syncthreads();
  fft_inplace<NN, false, RMAX>(d, nq, pitch, tws);
  float4 *Si = reinterpret_cast<float4 *>(S + (size_t)img * nh * n);
  for (int i = threadIdx.x; i < nh * nq; i += blockDim.x) {
    const int k = i / nq, q = i - k * nq;
    const float2 Z = d[q * pitch + fpad(k)], Zc = d[q * pitch + fpad((n - k) & (n - 1))];
    // row 2q: (Z + conj Zc)/2 ; row 2q+1: (Z - conj Zc)/(2i)
    float4 o;
    o.x = 0.5f * (Z.x + Zc.x);
    o.y = 0.5f * (Z.y - Zc.y);
    o.z = 0.5f * (Z.y + Zc.y);
    o.w = 0.5f * (Zc.x - Z.x);
    Si[((size_t)k * n + y0 + 2 * q) >> 1] = o;
  }
}

template <int NN, int RMAX>
__global__ void __launch_bounds__(kThreads)
k_cols(float2 *__restrict__ S, const float *__restrict__ kspec, int L,
       const float2 *__restrict__ tw, int tlen, int img0) {
  constexpr int n = NN, nh = (NN >> 1) + 1, CB = seqs_per_cta(NN);
  constexpr int pitch = n + (n >> 4);
  extern __shared__ float2 sm2[];
  const int img = blockIdx.y, band = (img0 + img) % L;
  const int k0 = blockIdx.x * CB;
  const int ncol = min(CB, nh - k0);
  float2 *d = sm2, *tws = sm2 + CB * pitch;
  load_tw(tws, tw, tlen);
  // element u of the thread is i = tid + 256 u of the CTA's [CB][n] block:
  // column c0 + 256 u / n, row tid % n + (256 u) % n (see k_rows_fwd)
  const int tid = threadIdx.x;
  const int c0 = tid / n, sb = c0 * pitch + fpad(tid % n);
  float2 *Si = S + ((size_t)img * nh + k0) * n + tid;
  const float *Ki = kspec + ((size_t)band * nh + k0) * n + tid;
  // every thread owns at most KPT multiplier entries: prefetch them now
  constexpr int KPT = NN < 16 ? NN : 16;
  float kr[KPT];
#pragma unroll
  for (int u = 0; u < KPT; ++u)
    kr[u] = c0 + (kThreads * u) / n < ncol ? __ldg(Ki + kThreads * u) : 0.f;
  {
    float2 v[KPT];
#pragma unroll
    for (int u = 0; u < KPT; ++u)
      if (c0 + (kThreads * u) / n < ncol) v[u] = Si[kThreads * u];
#pragma unroll
    for (int u = 0; u < KPT; ++u)
      if (c0 + (kThreads * u) / n < ncol)
        d[sb + ((kThreads * u) / n) * pitch + fpad((kThreads * u) % n)] = v[u];
  }
  __syncthreads();
  fft_inplace<NN, false, RMAX>(d, ncol, pitch, tws);
#pragma unroll
  for (int u = 0; u < KPT; ++u) {
    if (c0 + (kThreads * u) / n < ncol) {
      float2 &z = d[sb + ((kThreads * u) / n) * pitch + fpad((kThreads * u) % n)];
      z.x *= kr[u];
      z.y *= kr[u];
    }
  }
  __syncthreads();
  fft_inplace<NN, true, RMAX>(d, ncol, pitch, tws);
#pragma unroll
  for (int u = 0; u < KPT; ++u)
    if (c0 + (kThreads * u) / n < ncol)
      Si[kThreads * u] = d[sb + ((kThreads * u) / n) * pitch + fpad((kThreads * u) % n)];
}

template <int NN, int RMAX>
__global__ void __launch_bounds__(kThreads)
k_rows_inv(const float2 *__restrict__ S, float *__restrict__ g,
           const float *__restrict__ bdata, int L,
           const float2 *__restrict__ tw, int tlen, int img0) {
  constexpr int n = NN, nq = row_pairs(NN), nh = (NN >> 1) + 1, half = NN >> 1;
  constexpr int pitch = n + (n >> 4);
  extern __shared__ float2 sm2[];
  const int img = blockIdx.y, gimg = img0 + img, band = gimg % L;
  const int y0 = blockIdx.x * 2 * nq;
  float2 *d = sm2, *tws = sm2 + nq * pitch;
  load_tw(tws, tw, tlen);
  const float4 *Si = reinterpret_cast<const float4 *>(S + (size_t)img * nh * n);
  for (int i = threadIdx.x; i < nh * nq; i += blockDim.x) {
    const int k = i / nq, q = i - k * nq;
    float4 v = Si[((size_t)k * n + y0 + 2 * q) >> 1];   // Xa = (x,y), Xb = (z,w)
    if (k == 0 || k == half) { v.y = 0.f; v.w = 0.f; }
    d[q * pitch + fpad(k)] = make_float2(v.x - v.w, v.y + v.z);    // Xa + i Xb
    if (k > 0 && k < half)
      d[q * pitch + fpad(n - k)] = make_float2(v.x + v.w, v.z - v.y);  // conj Xa + i conj Xb
  }
  __syncthreads();
  fft_inplace<NN, true, RMAX>(d, nq, pitch, tws);
  const bool sub = (bdata != nullptr) && (gimg < L);
  // element u of the thread: row pair tid / n + 256 u / n (see k_rows_fwd)
  const int tid = threadIdx.x;
  const size_t o0 = (size_t)(y0 + 2 * (tid / n)) * n + tid % n;
  float *gi = g + (size_t)gimg * n * n + o0;
  const float *bi = sub ? bdata + (size_t)band * n * n + o0 : nullptr;
  const int sb = (tid / n) * pitch + fpad(tid % n);
  constexpr int VPT = fft_vpt(NN);
#pragma unroll
  for (int u = 0; u < VPT; ++u) {
    if (tid + u * kThreads >= nq * n) continue;
    const int q = (kThreads * u) / n, c = (kThreads * u) % n;
    const float2 z = d[sb + q * pitch + fpad(c)];
    float v0 = z.x, v1 = z.y;
    if (sub) {
      v0 -= __ldg(bi + 2 * q * n + c);
      v1 -= __ldg(bi + (2 * q + 1) * n + c);
    }
    gi[2 * q * n + c] = v0;
    gi[(2 * q + 1) * n + c] = v1;
  }
}

// ---------------------------------------------------------------- FP64 set-up
__global__ void k_fft64_rows(double2 *data, int n, bool inverse,
                             const double2 *__restrict__ tw) {
  extern __shared__ double2 sm4[];
  double2 *a = sm4, *b = sm4 + n;
  double2 *row = data + ((size_t)blockIdx.y * n + blockIdx.x) * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = row[i];
  __syncthreads();
  const double2 *r = inverse ? fft_batch<double2, true>(a, b, n, 1, tw)
                             : fft_batch<double2, false>(a, b, n, 1, tw);
  for (int i = threadIdx.x; i < n; i += blockDim.x) row[i] = r[i];
}

__global__ void k_transpose64(const double2 *__restrict__ in,
                              double2 *__restrict__ out, int n) {
  __shared__ double2 tile[32][33];
  const size_t base = (size_t)blockIdx.z * n * n;
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int y = by + j, x = bx + threadIdx.x;
    if (y < n && x < n) tile[j][threadIdx.x] = in[base + (size_t)y * n + x];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int y = bx + j, x = by + threadIdx.x;
    if (y < n && x < n) out[base + (size_t)y * n + x] = tile[threadIdx.x][j];
  }
}

__global__ void k_real_to_c64(const float *__restrict__ in,
                              double2 *__restrict__ out, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_double2((double)in[i], 0.0);
}

__global__ void k_mul_conj_c64(double2 *__restrict__ a,
                               const double2 *__restrict__ h, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    a[i] = cmulc(a[i], h[i]);
}

__global__ void k_c64_real_to_f32(const double2 *__restrict__ in,
                                  float *__restrict__ out, double scale,
                                  size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)(in[i].x * scale);
}

__global__ void k_make_kspec(const double2 *__restrict__ hh,
                             float *__restrict__ kspec, double scale, int n,
                             int L) {
  const int nh = (n >> 1) + 1;
  const size_t total = (size_t)L * nh * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int ky = (int)(i % n);
    const size_t r = i / n;
    const int kx = (int)(r % nh);
    const int l = (int)(r / nh);
    const double2 h = hh[((size_t)l * n + ky) * n + kx];
    kspec[i] = (float)((h.x * h.x + h.y * h.y) * scale);
  }
}

inline int grid_for(size_t count) {
  size_t g = (count + 255) / 256;
  return (int)(g > 152 * 32 ? 152 * 32 : (g ? g : 1));
}


template <int NN, int RMAX>
cudaError_t gradient_n(const float *x, float *g, const float *b, float2 *S,
                       const float *kspec, const float2 *tw, int L, int C,
                       cudaStream_t st, Prof *prof, int chunk) {
  constexpr int n = NN;
  const int ntot = C * L;
  const int RB = 2 * row_pairs(n);                  // real rows per CTA (even)
  const int CB = seqs_per_cta(n);                   // columns per CTA
  const int nh = (n >> 1) + 1;
  const int pitch = n + (n >> 4);
  const int tlen = fft_table_len(n, RMAX);
  const size_t smr = ((size_t)(RB / 2) * pitch + tlen) * sizeof(float2);
  const size_t smc = ((size_t)CB * pitch + tlen) * sizeof(float2);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rows_fwd<NN, RMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_rows_inv<NN, RMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_cols<NN, RMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const double img = (double)n * n, spec = (double)nh * n * 8.0;
  const double fft = 5.0 * n * ilog2(n);   // flops of one length-n complex FFT
  const int step = chunk > 0 && chunk < ntot ? chunk : ntot;
  // the whole call: x read, g written, b read, |h_hat|^2 read once per
  // band, the spectra of every image written and read twice
  ProfScope all(prof, "grad_total",
                ntot * (img * 8.0 + 4.0 * spec) + (b ? (double)L * img * 4.0 : 0.0) +
                    (double)L * nh * n * 4.0,
                ntot * (double)(n + 2 * nh) * fft, st);
  for (int i0 = 0; i0 < ntot; i0 += step) {
    const int nimg = step < ntot - i0 ? step : ntot - i0;
    const int nb = b ? (i0 < L ? (L - i0 < nimg ? L - i0 : nimg) : 0) : 0;   // images with b
    {
      ProfScope ps(prof, "grad_rows_fwd", nimg * (img * 4.0 + spec),
                   nimg * (n / 2.0) * fft, st);
      k_rows_fwd<NN, RMAX><<<dim3(n / RB, nimg), kThreads, smr, st>>>(x, S, tw, tlen, i0);
    }
    {
      ProfScope ps(prof, "grad_cols", nimg * 2.0 * spec + (double)nimg * nh * n * 4.0,
                   nimg * (double)nh * 2.0 * fft, st);
      k_cols<NN, RMAX><<<dim3((nh + CB - 1) / CB, nimg), kThreads, smc, st>>>(S, kspec, L, tw, tlen, i0);
    }
    {
      ProfScope ps(prof, "grad_rows_inv", nimg * (spec + img * 4.0) + nb * img * 4.0,
                   nimg * (n / 2.0) * fft, st);
      k_rows_inv<NN, RMAX><<<dim3(n / RB, nimg), kThreads, smr, st>>>(S, g, b, L, tw, tlen, i0);
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gradient(const float *x, float *g, const float *b,
                            float2 *S, const float *kspec, const float2 *tw,
                            int n, int L, int C, cudaStream_t st, Prof *prof, int chunk,
                            int radix) {
  const bool r8 = radix == 8 && n >= 64;   // the alternative plan exists from n = 64
#define MUFFIN_GRAD(NN)                                                                    \
  return r8 ? gradient_n<NN, 8>(x, g, b, S, kspec, tw, L, C, st, prof, chunk)              \
            : gradient_n<NN, 16>(x, g, b, S, kspec, tw, L, C, st, prof, chunk)
#define MUFFIN_GRAD16(NN) return gradient_n<NN, 16>(x, g, b, S, kspec, tw, L, C, st, prof, chunk)
  switch (n) {
    case 2: MUFFIN_GRAD16(2);
    case 4: MUFFIN_GRAD16(4);
    case 8: MUFFIN_GRAD16(8);
    case 16: MUFFIN_GRAD16(16);
    case 32: MUFFIN_GRAD16(32);
    case 64: MUFFIN_GRAD(64);
    case 128: MUFFIN_GRAD(128);
    case 256: MUFFIN_GRAD(256);
    case 512: MUFFIN_GRAD(512);
    case 1024: MUFFIN_GRAD(1024);
    case 2048: MUFFIN_GRAD(2048);
#undef MUFFIN_GRAD
#undef MUFFIN_GRAD16
    default: return cudaErrorInvalidValue;
  }
}

int fft32_table_len(int n, int radix) { return fft_table_len(n, radix); }
void fft32_tables(int n, float2 *tab, int radix) { fft_tables(n, tab, radix); }

cudaError_t fft2d_c64(double2 *data, double2 *tmp, int n, int nimg,
                      bool inverse, const double2 *tw64, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_fft64_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const size_t sm = (size_t)2 * n * sizeof(double2);
  const int thr = n < 256 ? (n < 32 ? 32 : n) : 256;
  dim3 tg((n + 31) / 32, (n + 31) / 32, nimg), tb(32, 8);
  k_fft64_rows<<<dim3(n, nimg), thr, sm, st>>>(data, n, inverse, tw64);
  k_transpose64<<<tg, tb, 0, st>>>(data, tmp, n);
  k_fft64_rows<<<dim3(n, nimg), thr, sm, st>>>(tmp, n, inverse, tw64);
  k_transpose64<<<tg, tb, 0, st>>>(tmp, data, n);
  return cudaGetLastError();
}

cudaError_t real_to_c64(const float *in, double2 *out, size_t count,
                        cudaStream_t st) {
  k_real_to_c64<<<grid_for(count), 256, 0, st>>>(in, out, count);
  return cudaGetLastError();
}

cudaError_t mul_conj_c64(double2 *a, const double2 *h, size_t count,
                         cudaStream_t st) {
  k_mul_conj_c64<<<grid_for(count), 256, 0, st>>>(a, h, count);
  return cudaGetLastError();
}

cudaError_t c64_real_to_f32(const double2 *in, float *out, double scale,
                            size_t count, cudaStream_t st) {
  k_c64_real_to_f32<<<grid_for(count), 256, 0, st>>>(in, out, scale, count);
  return cudaGetLastError();
}

cudaError_t make_kspec(const double2 *hh, float *kspec, double scale, int n,
                       int L, cudaStream_t st) {
  const size_t total = (size_t)L * ((n >> 1) + 1) * n;
  k_make_kspec<<<grid_for(total), 256, 0, st>>>(hh, kspec, scale, n, L);
  return cudaGetLastError();
}

}  // namespace muffin
