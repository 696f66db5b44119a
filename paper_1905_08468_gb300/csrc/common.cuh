// Shared device-side definitions of the MUFFIN CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace muffin {

// Device-resident iteration scalars.  The ADA-PT update kernel rewrites mu,
// gamma and tau in place, so captured launch sequences stay valid.
struct DevScalars {
  double mu;      // spatial weight mu (theta[0])
  double gamma;   // spectral weight gamma (theta[1])
  double tau;     // primal step
  double sigma;   // dual step
};

// One group of chains advanced by the same fused kernels.  C = 1: a plain
// MUFFIN chain.  C = 3: an ADA-PT group {primal, d/dmu, d/dgamma} that
// shares the masks of its primal (Algorithms 3 and 4).
struct Group {
  int C;
  float *x;    // [C][L][n][n] current primal x (= x-tilde of the last step)
  float *xt;   // [C][L][n][n] next primal x-tilde
  float *u;    // [C][L][K][n][n] spatial duals (Mallat layout per basis)
  float *v;    // [C][L][n][n] spectral duals (band index = DCT index)
  float *t;    // [C][L][n][n] spectral back-projection t = gamma_n C^T v
  float *g;    // [C][L][n][n] least-squares gradient
  const float *b;  // [L][n][n] H^T y of this group's data (chain 0 only)
};

__host__ __device__ inline int ilog2(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

__device__ __forceinline__ float satf(float p) {
  return fminf(fmaxf(p, -1.0f), 1.0f);
}

}  // namespace muffin
