// ccg_matvec_h_noalloc: y = A^H x for a dense matrix without any device
// allocation, for callers that cannot call cudaMalloc (see include/ccg.h).
//
// The column-tiled sweep (gemv.cuh, gemv_tile) leaves one partial vector per
// row range; here those partials live in a fixed file-scope device array
// instead of a handle's workspace, and a small kernel sums them into y.
// The array is resident on a device from the first call there (or from
// library load under eager module loading) until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "common.cuh"
#include "gemv.cuh"
#include "internal.h"

namespace ccg {
namespace {

constexpr size_t kScratchBytes = size_t(CCG_NOALLOC_SCRATCH_BYTES);
constexpr int kMaxDevices = 64;

// Partial sums of the sweep.  Shared by every call on a device; each call
// overwrites every entry it later reads, so nothing needs clearing.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

template <class R>
__global__ void __launch_bounds__(kBlock) sum_partials(const cx<R>* __restrict__ P, int nparts, int64_t n,
                                                       cx<R>* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
    cx<R> s = P[i];
    for (int q = 1; q < nparts; ++q) s = cadd(s, P[(int64_t)q * n + i]);
    y[i] = s;
  }
}

struct DeviceSetup {
  bool ready = false;
  void* scratch = nullptr;  // device address of g_scratch on this device
  int num_sms = 1;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

// Once per device, with that device current: look up the device address of
// the scratch array (the host-side symbol is only a stand-in).
int setup_current_device(DeviceSetup** out) {
  int count = 0, dev = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    set_error("ccg_matvec_h_noalloc: no CUDA device");
    return CCG_ERR_CUDA;
  }
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    set_error("ccg_matvec_h_noalloc: cannot use the current device");
    return CCG_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      set_error(std::string("ccg_matvec_h_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return CCG_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
      cudaGetLastError();
      sms = 1;
    }
    // Load every kernel this entry point can launch now, so that under lazy
    // module loading no later call (of either precision or load width)
    // loads a kernel, e.g. inside a stream capture.
    const void* kernels[] = {(const void*)gemv_tile_h<double, 1, 4>, (const void*)gemv_tile_h<float, 1, 4>,
                             (const void*)gemv_tile_h<float, 2, 4>, (const void*)sum_partials<double>,
                             (const void*)sum_partials<float>};
    for (const void* k : kernels) {
      cudaFuncAttributes attr;
      const cudaError_t ek = cudaFuncGetAttributes(&attr, k);
      if (ek != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("ccg_matvec_h_noalloc: cannot load a kernel: ") + cudaGetErrorString(ek));
        return CCG_ERR_CUDA;
      }
    }
    s.scratch = p;
    s.num_sms = sms;
    s.ready = true;
  }
  *out = &s;
  return CCG_OK;
}

template <class R>
int run(const DeviceSetup& dev, int64_t n, const void* A_, int64_t lda, const void* x_, void* y_, int unit,
        cudaStream_t stream) {
  constexpr int E = 4;
  const cx<R>* A = static_cast<const cx<R>*>(A_);
  const cx<R>* x = static_cast<const cx<R>*>(x_);
  cx<R>* y = static_cast<cx<R>*>(y_);
  cx<R>* P = static_cast<cx<R>*>(dev.scratch);
  // Same launch shape as the handle path's A^H x sweep, with fewer row ranges
  // if their partials would not fit the scratch array.
  const int64_t nunits = n / unit;
  const int ncb = (int)((nunits + 32 * E - 1) / (32 * E));
  int64_t ns = ((int64_t)dev.num_sms * 4 + ncb - 1) / ncb;
  ns = ns < 1 ? 1 : ns;
  const int64_t cap_rows = (n + kWarps - 1) / kWarps;
  ns = ns > 32 ? 32 : ns;
  ns = ns > cap_rows ? cap_rows : ns;
  // Guard for GPUs with many more SMs: on 152 SMs ns * n stays below
  // 4 * 152 * 128 + n (about 0.2 M elements at the n cap), far inside the
  // array, so this never trims there.
  while (ns > 1 && (size_t)ns * (size_t)n * sizeof(cx<R>) > kScratchBytes) --ns;
  const int64_t rows_per_range = (n + ns - 1) / ns;
  const int nsplit = (int)((n + rows_per_range - 1) / rows_per_range);
  dim3 grid(ncb, nsplit);
  if (unit == 2) {
    if constexpr (sizeof(R) == 4)
      gemv_tile_h<R, 2, E><<<grid, kBlock, 0, stream>>>(A, lda, n, rows_per_range, x, P,
                                                                   nullptr);
  } else {
    gemv_tile_h<R, 1, E><<<grid, kBlock, 0, stream>>>(A, lda, n, rows_per_range, x, P,
                                                                 nullptr);
  }
  int gsum = (int)((n + kBlock - 1) / kBlock);
  gsum = gsum > dev.num_sms * 8 ? dev.num_sms * 8 : gsum;
  sum_partials<R><<<gsum, kBlock, 0, stream>>>(P, nsplit, n, y);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("ccg_matvec_h_noalloc: launch failed: ") + cudaGetErrorString(e));
    return CCG_ERR_CUDA;
  }
  return CCG_OK;
}

bool is_aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace
}  // namespace ccg

extern "C" ccg_status ccg_matvec_h_noalloc(ccg_dtype dtype, int64_t n, const void* A, int64_t lda, const void* x,
                                           void* y, void* stream) {
  using namespace ccg;
  if (!A || !x || !y) { set_error("ccg_matvec_h_noalloc: NULL pointer"); return CCG_ERR_INVALID; }
  if (dtype != CCG_C64 && dtype != CCG_C128) { set_error("ccg_matvec_h_noalloc: bad dtype"); return CCG_ERR_INVALID; }
  if (n < 1 || lda < n) { set_error("ccg_matvec_h_noalloc: need n >= 1 and lda >= n"); return CCG_ERR_INVALID; }
  if (n > CCG_NOALLOC_MAX_N) {
    set_error("ccg_matvec_h_noalloc: n = " + std::to_string(n) + " exceeds the maximum " +
              std::to_string((long long)CCG_NOALLOC_MAX_N) + " of the fixed scratch array");
    return CCG_ERR_INVALID;
  }
  const size_t esz = dtype == CCG_C128 ? 16 : 8;
  if (!is_aligned(A, esz) || !is_aligned(x, esz) || !is_aligned(y, esz)) {
    set_error("ccg_matvec_h_noalloc: pointer not aligned to the element size");
    return CCG_ERR_INVALID;
  }
  DeviceSetup* dev = nullptr;
  const int rc = setup_current_device(&dev);
  if (rc != CCG_OK) return static_cast<ccg_status>(rc);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == CCG_C128) return static_cast<ccg_status>(run<double>(*dev, n, A, lda, x, y, 1, s));
  const int unit = (n % 2 == 0 && lda % 2 == 0 && is_aligned(A, 16) && is_aligned(x, 16)) ? 2 : 1;
  return static_cast<ccg_status>(run<float>(*dev, n, A, lda, x, y, unit, s));
}
