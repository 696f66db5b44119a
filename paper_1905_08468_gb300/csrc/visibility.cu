// Visibility-domain data term (Sec. 1: the method runs unchanged with a
// direct operator that maps the sky to the visibilities).  Reading:
// visibilities sample the unitary 2D DFT U = F / n of each band on the n x n
// grid and are gridded into per-cell sums D_l[k] and natural weights m_l[k];
// for real x the gradient of 1/2 sum_p |d_p - (U x_l)_{k(p)}|^2 is
//   F^-1 (m~_l . F x_l) - Re U^H D_l,    m~_l[k] = (m_l[k] + m_l[-k]) / 2,
// the image-domain gradient with |h_hat_l|^2 = m~_l and H^T y = Re U^H D_l.
// These kernels turn (D, m) into the plan's FP64 spectra h_hat = sqrt(m~)
// and the complex input of the FP64 inverse DFT that yields b.
#include <cuda_runtime.h>

#include "kernels.h"

namespace muffin {

namespace {

// h_hat = (sqrt(m~), 0); chk = m with NaN where m < 0 (for the input scan)
__global__ void k_vis_weights(const float *__restrict__ m, double2 *__restrict__ hh,
                              float *__restrict__ chk, int n, size_t nimg) {
  const size_t N = (size_t)n * n, total = N * nimg;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t img = i / N, r = i - img * N;
    const int ky = (int)(r / n), kx = (int)(r - (size_t)ky * n);
    const size_t mi = img * N + (size_t)((n - ky) & (n - 1)) * n + ((n - kx) & (n - 1));
    const float a = m[i], b = m[mi];
    const double ms = 0.5 * ((double)a + (double)b);
    hh[i] = make_double2(ms > 0.0 ? sqrt(ms) : 0.0, 0.0);
    chk[i] = a >= 0.f ? a : __int_as_float(0x7fc00000);
  }
}

__global__ void k_vis_c64(const float2 *__restrict__ in, double2 *__restrict__ out,
                          size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = in[i];
    out[i] = make_double2(v.x, v.y);
  }
}

int grid_of(size_t count) {
  const size_t g = (count + 255) / 256;
  return (int)(g > 152 * 32 ? 152 * 32 : (g ? g : 1));
}

}  // namespace

cudaError_t vis_weights(const float *m, double2 *hh, float *chk, int n, int nimg,
                        cudaStream_t st) {
  k_vis_weights<<<grid_of((size_t)n * n * nimg), 256, 0, st>>>(m, hh, chk, n, (size_t)nimg);
  return cudaGetLastError();
}

cudaError_t vis_to_c64(const float *vis, double2 *out, size_t count, cudaStream_t st) {
  k_vis_c64<<<grid_of(count), 256, 0, st>>>(reinterpret_cast<const float2 *>(vis), out, count);
  return cudaGetLastError();
}

}  // namespace muffin
