// Allocation-free entry point: the spatial analysis operator u = W_s x
// (the same kernels as muffin_op_analysis) without a plan and without any
// device allocation.  Levels 2..J of the transform need an LL scratch; here
// it is a fixed file-scope device array instead of plan-owned memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/muffin.h"
#include "host_math.h"
#include "kernels.h"

// Maximum LL scratch, in floats: 4 Mi floats = 16 MiB, held by every GPU
// that loads the library until the process exits.
static constexpr size_t kNoAllocScratchFloats = size_t(4) << 20;
static __device__ __align__(256) float g_noalloc_ll[kNoAllocScratchFloats];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float *g_ll_dev[kMaxDevices] = {};            // device address of g_noalloc_ll per device
unsigned long long g_ctx_id[kMaxDevices] = {}; // context the set-up was done in

muffin_status noalloc_fail(muffin_status s, const char *m) {
  return static_cast<muffin_status>(muffin::set_last_error_code(s, m));
}

// memory the current device `dev` can dereference: its own device memory or
// managed memory (device memory of another GPU would need peer access)
bool usable_on(const void *p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// unique id of the current context (cuCtxGetId never reuses an id), so a
// set-up done before a cudaDeviceReset is detected and redone; 0 if the
// driver does not provide it
unsigned long long current_context_id() {
  using GetCur = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static GetCur get_cur = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<GetCur>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_cur || !get_id || get_cur(&ctx) != CUDA_SUCCESS || !ctx ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

bool overlap(const void *a, size_t na, const void *b, size_t nb) {
  const uintptr_t pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
  return pa < pb + nb && pb < pa + na;
}

}  // namespace

extern "C" MUFFIN_API muffin_status muffin_op_analysis_noalloc(
    const float *x, float *u, int32_t n, int32_t nbands, int32_t n_wavelets,
    int32_t levels, void *stream) {
  using namespace muffin;
  if (!x || !u) return noalloc_fail(MUFFIN_EINVAL, "x and u must be non-NULL");
  if (n < 2 || n > 2048 || (n & (n - 1)))
    return noalloc_fail(MUFFIN_EINVAL, "n must be a power of two in [2, 2048]");
  if (nbands < 1 || n_wavelets < 1 || n_wavelets > 8)
    return noalloc_fail(MUFFIN_EINVAL, "nbands >= 1 and 1 <= n_wavelets <= 8 required");
  if (levels < 0 || levels > 15 || (1 << levels) > n)
    return noalloc_fail(MUFFIN_EINVAL, "levels must satisfy 2^levels <= n");
  // LL scratch of levels 1..J-1: [L][K][n>>j][n>>j]
  WaveArgs w{};
  size_t need = 0;
  for (int j = 1; j < levels; ++j) {
    w.lvl_off[j] = need;
    const size_t h = (size_t)(n >> j);
    need += (size_t)nbands * n_wavelets * h * h;
  }
  if (need > kNoAllocScratchFloats)
    return noalloc_fail(MUFFIN_EINVAL,
                        "cube too large for the fixed scratch (needs nbands * n_wavelets * "
                        "sum_{1<=j<levels} (n>>j)^2 <= 4194304 floats)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return noalloc_fail(MUFFIN_ECUDA, "no usable current CUDA device");
  }
  if (!usable_on(x, dev) || !usable_on(u, dev))
    return noalloc_fail(MUFFIN_EINVAL,
                        "x and u must be device (or managed) arrays of the current device");
  const size_t xbytes = (size_t)nbands * n * n * sizeof(float);
  if (overlap(x, xbytes, u, xbytes * n_wavelets))
    return noalloc_fail(MUFFIN_EINVAL, "x and u must not overlap");
  {
    // once per device (and again if its context was reset), with that device
    // current: the scratch's device address (the host-side name is only a
    // stand-in) and the filter taps
    std::lock_guard<std::mutex> lk(g_setup_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_ll_dev[dev] || ctx != g_ctx_id[dev]) {
      g_ll_dev[dev] = nullptr;
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_ll) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return noalloc_fail(MUFFIN_ECUDA, "cudaGetSymbolAddress of the scratch failed");
      }
      double taps[8][16];
      std::memset(taps, 0, sizeof(taps));
      for (int p = 1; p <= 8; ++p) daubechies_lowpass(p, taps[p - 1]);
      if (upload_filters(taps) != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(MUFFIN_ECUDA, "filter upload failed");
      }
      g_ll_dev[dev] = static_cast<float *>(ptr);
      g_ctx_id[dev] = ctx;
    }
  }
  w.n = n; w.L = nbands; w.K = n_wavelets; w.J = levels; w.C = 1;
  w.scratch = g_ll_dev[dev];
  w.beta = nullptr; w.sc = nullptr; w.prof = nullptr;
  const cudaError_t e = wavelet_analysis_op(w, x, u, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return noalloc_fail(MUFFIN_ECUDA, cudaGetErrorString(e));
  return MUFFIN_OK;
}
