// FP32 in-place shared-memory FFT of the gradient passes (hot path).
//
// A batch of nb length-N sequences (N a power of two) lives in shared memory
// in a padded layout (element i of a sequence at i + i/16, which makes the
// stride-16 stores of the first stage bank-conflict free).  Every thread owns
// VPT = min(16, N) complex values per stage: radix-RMAX stages while at
// least RMAX points remain, then one smaller stage (RMAX = 16, the default
// plan: N = 1024 is 16, 16, 4; RMAX = 8, the alternative plan the tuner may
// pick: 8, 8, 8, 2, each thread running two radix-8 butterflies per stage).
// A stage is the Stockham step  out[(j-k) R + k + r Ns] = DFT_R(w^{kr} in[j +
// r N/R]); it reads, synchronises, then writes in place.  Stage twiddles
// w = exp(-2 pi i k r / (Ns R)) come from a host-computed table laid out
// [r-1][k] per stage, staged in shared memory by the calling kernel.
#pragma once

#include "fft.cuh"

namespace muffin {

__device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }

template <bool INV>
__device__ __forceinline__ float2 twid(float2 v, float2 w) {
  return INV ? cmulc(v, w) : cmul(v, w);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2 &a, float2 &b) {
  const float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
  const float2 s02 = cadd(x0, x2), d02 = csub(x0, x2);
  const float2 s13 = cadd(x1, x3), d13 = crot<float2, INV>(csub(x1, x3));
  x0 = cadd(s02, s13);
  x1 = cadd(d02, d13);
  x2 = csub(s02, s13);
  x3 = csub(d02, d13);
}

// W_M^e (forward sign) for the in-register sub-transforms
template <bool INV>
__device__ __forceinline__ float2 wmul(float2 v, float c, float s) {
  // multiply by (c - i s) forward, (c + i s) inverse
  float2 r;
  if (INV) { r.x = v.x * c - v.y * s; r.y = v.x * s + v.y * c; }
  else { r.x = v.x * c + v.y * s; r.y = v.y * c - v.x * s; }
  return r;
}

// radix-8 = 2 x 4: x[n], n = 4 n1 + n2 (n1 < 2, n2 < 4); X[k1 + 2 k2]
template <bool INV>
__device__ __forceinline__ void dft8(float2 *v) {
  const float h = 0.70710678118654752f;
  // DFT2 over n1 for every n2
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft2<INV>(v[n2], v[4 + n2]);
  // twiddle W8^{n2 k1}: k1 = 1 row is v[4 + n2]
  v[5] = wmul<INV>(v[5], h, h);
  v[6] = crot<float2, INV>(v[6]);
  v[7] = wmul<INV>(v[7], -h, h);
  // DFT4 over n2 for every k1
  dft4<INV>(v[0], v[1], v[2], v[3]);
  dft4<INV>(v[4], v[5], v[6], v[7]);
  // X[k1 + 2 k2] is left in v[4 k1 + k2] (see out_slot)
}

// radix-16 = 4 x 4: x[n], n = 4 n1 + n2; X[k1 + 4 k2]
template <bool INV>
__device__ __forceinline__ void dft16(float2 *v) {
  const float c1 = 0.92387953251128676f, s1 = 0.38268343236508977f;
  const float h = 0.70710678118654752f;
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
  // row k1 holds v[4 k1 + n2]; twiddle W16^{n2 k1}
  v[5] = wmul<INV>(v[5], c1, s1);
  v[6] = wmul<INV>(v[6], h, h);
  v[7] = wmul<INV>(v[7], s1, c1);
  v[9] = wmul<INV>(v[9], h, h);
  v[10] = crot<float2, INV>(v[10]);
  v[11] = wmul<INV>(v[11], -h, h);
  v[13] = wmul<INV>(v[13], s1, c1);
  v[14] = wmul<INV>(v[14], -h, h);
  v[15] = wmul<INV>(v[15], -c1, -s1);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
    dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // X[k1 + 4 k2] is left in v[4 k1 + k2] (see out_slot)
}

// register slot holding output r of dftR
template <int R>
__device__ __forceinline__ constexpr int out_slot(int r) {
  return R == 16 ? 4 * (r & 3) + (r >> 2) : (R == 8 ? 4 * (r & 1) + (r >> 1) : r);
}

template <int R, bool INV>
__device__ __forceinline__ void dftR(float2 *v) {
  if (R == 16) dft16<INV>(v);
  else if (R == 8) dft8<INV>(v);
  else if (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else dft2<INV>(v[0], v[1]);
}

// one Stockham stage of radix R (N and Ns fixed at compile time); every
// active thread handles VPT/R butterflies
template <int N, int NS, int R, int VPT, bool INV>
__device__ __forceinline__ void fft_stage(float2 *d, int pitch, int nthr,
                                          const float2 *tw) {
  constexpr int G = VPT / R;
  constexpr int q = N / R;
  const int tid = threadIdx.x;
  const bool act = tid < nthr;
  float2 v[VPT];
  if (act) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int w = tid + g * nthr;
      const int s = w / q, j = w % q, k = j & (NS - 1);
      const float2 *src = d + s * pitch;
      if constexpr (q % 16 == 0) {
        // j + r q and j share their position within a 16-run: one base
        // address, constant offsets
        const float2 *b = src + fpad(j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[g * R + r] = b[r * (q + q / 16)];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[g * R + r] = src[fpad(j + r * q)];
      }
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r)
          v[g * R + r] = twid<INV>(v[g * R + r], tw[(r - 1) * NS + k]);
      }
      dftR<R, INV>(v + g * R);
    }
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int w = tid + g * nthr;
      const int s = w / q, j = w % q, k = j & (NS - 1);
      float2 *dst = d + s * pitch;
      const int o = (j - k) * R + k;
      if constexpr (NS % 16 == 0 || (NS == 1 && (R == 16 || N <= 16))) {
        // o + r NS stays in o's 16-run (NS = 1: o is a multiple of R = 16,
        // or o = 0 for N <= 16) or moves by whole runs (NS a multiple of 16)
        float2 *b = dst + fpad(o);
#pragma unroll
        for (int r = 0; r < R; ++r) b[r * (NS + NS / 16)] = v[g * R + out_slot<R>(r)];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) dst[fpad(o + r * NS)] = v[g * R + out_slot<R>(r)];
      }
    }
  }
  __syncthreads();
}

__host__ __device__ constexpr int fft_vpt(int N) { return N < 16 ? N : 16; }

template <int N, int NS, bool INV, int RMAX>
__device__ __forceinline__ void fft_stages(float2 *d, int pitch, int nthr,
                                           const float2 *tw) {
  if constexpr (NS < N) {
    constexpr int REM = N / NS;
    constexpr int R = REM >= RMAX ? RMAX : REM;
    fft_stage<N, NS, R, fft_vpt(N), INV>(d, pitch, nthr, tw);
    fft_stages<N, NS * R, INV, RMAX>(d, pitch, nthr, tw + (NS > 1 ? (R - 1) * NS : 0));
  }
}

// In-place transform of nb sequences (sequence s at d + s * pitch, padded
// layout).  Needs nb * N / fft_vpt(N) <= blockDim.x.  Caller syncs before.
template <int N, bool INV, int RMAX = 16>
__device__ __forceinline__ void fft_inplace(float2 *d, int nb, int pitch,
                                            const float2 *tws) {
  fft_stages<N, 1, INV, RMAX>(d, pitch, nb * N / fft_vpt(N), tws);
}

// number of complex entries of the stage twiddle tables for N
inline int fft_table_len(int N, int rmax = 16) {
  if (N < 16) return 1;
  int Ns = 1, len = 0;
  while (Ns < N) {
    const int rem = N / Ns;
    const int R = rem >= rmax ? rmax : rem;
    if (Ns > 1) len += (R - 1) * Ns;
    Ns *= R;
  }
  return len > 0 ? len : 1;
}

// fills tab[fft_table_len(N, rmax)] in the order the stages read it
inline void fft_tables(int N, float2 *tab, int rmax = 16) {
  const double pi = 3.14159265358979323846;
  if (N < 16) { tab[0] = make_float2(1.f, 0.f); return; }
  int Ns = 1, off = 0;
  while (Ns < N) {
    const int rem = N / Ns;
    const int R = rem >= rmax ? rmax : rem;
    if (Ns > 1) {
      for (int r = 1; r < R; ++r)
        for (int k = 0; k < Ns; ++k) {
          const double a = -2.0 * pi * (double)k * r / ((double)Ns * R);
          tab[off + (r - 1) * Ns + k] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
      off += (R - 1) * Ns;
    }
    Ns *= R;
  }
}

}  // namespace muffin
