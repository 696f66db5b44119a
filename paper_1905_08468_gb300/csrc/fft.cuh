// Shared-memory Stockham FFT used by the convolution kernels.
//
// H_l = F^-1 diag(h_hat_l) F (circular convolution, Eq. model), so the
// least-squares gradient of Algorithm 2 (eq. grad2) needs forward and
// inverse 2D DFTs of every band.  The row and column passes below hold whole
// sequences in shared memory: a batch of nb sequences of length N (a power
// of two) is transformed in place with radix-4 stages (one radix-2 stage
// first when log2 N is odd), ping-ponging between two buffers.
#pragma once

#include "common.cuh"

namespace muffin {

template <typename C> struct Real;
template <> struct Real<float2> { using type = float; };
template <> struct Real<double2> { using type = double; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) {
  C r; r.x = a.x + b.x; r.y = a.y + b.y; return r;
}
template <typename C> __device__ __forceinline__ C csub(C a, C b) {
  C r; r.x = a.x - b.x; r.y = a.y - b.y; return r;
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
// multiply by -i (forward) or +i (inverse)
template <typename C, bool INV> __device__ __forceinline__ C crot(C a) {
  C r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

// Transforms nb sequences of length N stored at a[s*N .. s*N+N-1].
// Forward (INV=false): X[k] = sum_j x[j] exp(-2 pi i jk/N); inverse: the
// unnormalised conjugate transform.  tw[k] = exp(-2 pi i k/N), k < N.
// All threads of the block must call it; data must be visible in shared
// memory on entry (caller syncs).  Returns the buffer holding the result
// (a or b); the other one is free scratch.  Ends with __syncthreads().
template <typename C, bool INV>
__device__ C *fft_batch(C *a, C *b, int N, int nb, const C *__restrict__ tw) {
  const int logN = ilog2(N);
  int Ns = 1;
  if (logN & 1) {
    const int half = N >> 1;
    const int lh = logN - 1;
    for (int w = threadIdx.x; w < nb * half; w += blockDim.x) {
      const int s = w >> lh, j = w & (half - 1);
      const C *in = a + s * N;
      C *out = b + s * N;
      const C v0 = in[j], v1 = in[j + half];
      out[2 * j] = cadd(v0, v1);
      out[2 * j + 1] = csub(v0, v1);
    }
    __syncthreads();
    C *t = a; a = b; b = t;
    Ns = 2;
  }
  if (N >= 4) {
    const int q = N >> 2;
    const int lq = logN - 2;
    while (Ns < N) {
      const int tstride = N / (Ns * 4);
      for (int w = threadIdx.x; w < nb * q; w += blockDim.x) {
        const int s = w >> lq, j = w & (q - 1);
        const int k = j & (Ns - 1);
        const C *in = a + s * N;
        C *out = b + s * N;
        C v0 = in[j], v1 = in[j + q], v2 = in[j + 2 * q], v3 = in[j + 3 * q];
        if (Ns > 1) {
          const C w1 = tw[k * tstride], w2 = tw[2 * k * tstride],
                  w3 = tw[3 * k * tstride];
          if (INV) { v1 = cmulc(v1, w1); v2 = cmulc(v2, w2); v3 = cmulc(v3, w3); }
          else { v1 = cmul(v1, w1); v2 = cmul(v2, w2); v3 = cmul(v3, w3); }
        }
        const C s02 = cadd(v0, v2), d02 = csub(v0, v2);
        const C s13 = cadd(v1, v3), d13 = crot<C, INV>(csub(v1, v3));
        const int idx = ((j - k) << 2) + k;
        out[idx] = cadd(s02, s13);
        out[idx + Ns] = cadd(d02, d13);
        out[idx + 2 * Ns] = csub(s02, s13);
        out[idx + 3 * Ns] = csub(d02, d13);
      }
      __syncthreads();
      C *t = a; a = b; b = t;
      Ns <<= 2;
    }
  }
  return a;
}

}  // namespace muffin
