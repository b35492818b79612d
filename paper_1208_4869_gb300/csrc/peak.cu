// Measured issue rates of the arithmetic pipes the sweeps run on, so that a
// kernel bound by arithmetic is compared with what this GPU retires rather
// than with a datasheet figure: FP64 fused multiply-add (the complex128
// sweeps on the FP64 pipe), FP32 fused multiply-add, and the 32 x 32 -> 64-bit
// integer multiply-add of the fixed-point complex128 sweep (fx.cuh).
//
// Each thread runs 8 independent dependency chains (enough to cover the
// pipes' latency at 8 resident blocks of 256 threads per SM), on data the
// compiler cannot see, and stores its sums only under a condition that never
// holds, so no chain can be removed or folded.
#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"

namespace ccg {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) rate_dfma(const double* in, double* out, int iters) {
  const double a = in[threadIdx.x & 31], b = in[(threadIdx.x + 7) & 31];
  double c[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) c[k] = in[k];
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) c[k] = fma(a, b, c[k]);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k];
  if (s == 12345.0) out[0] = s;
}

__global__ void __launch_bounds__(256) rate_ffma(const float* in, float* out, int iters) {
  const float a = in[threadIdx.x & 31], b = in[(threadIdx.x + 7) & 31];
  float c[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) c[k] = in[k];
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) c[k] = fmaf(a, b, c[k]);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k];
  if (s == 12345.0f) out[0] = s;
}

// c += (int64) a * b, the accumulation of the fixed-point sweep.  An empty
// asm statement makes each multiplier opaque to the compiler every
// iteration (it emits no instruction), so no closed form of the sum can
// replace the loop.
__global__ void __launch_bounds__(256) rate_imad_wide(const int* in, long long* out, int iters) {
  const int b = in[threadIdx.x & 31];
  int a[kChains];
  long long c[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    a[k] = in[(threadIdx.x + k) & 31];
    c[k] = in[(threadIdx.x + k + 3) & 31];
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      c[k] += (long long)a[k] * b;
      asm volatile("" : "+r"(a[k]));
    }
  }
  long long s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k];
  if (s == 0x123456789ll) out[0] = s;
}

// The same product through the two explicit PTX forms of a 32 x 32 + 64
// multiply-add: FORM 0 mad.wide.s32, FORM 1 mad.lo.cc.u32 + madc.hi.s32.
template <int FORM>
__global__ void __launch_bounds__(256) rate_mad_ptx(const int* in, long long* out, int iters) {
  const int b = in[threadIdx.x & 31];
  int a[kChains];
  long long c[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    a[k] = in[(threadIdx.x + k) & 31];
    c[k] = in[(threadIdx.x + k + 3) & 31];
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      long long d;
      if (FORM == 0) {
        asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a[k]), "r"(b), "l"(c[k]));
      } else {
        asm("{\n\t.reg .u32 cl, ch, dl, dh;\n\tmov.b64 {cl, ch}, %3;\n\t"
            "mad.lo.cc.u32 dl, %1, %2, cl;\n\tmadc.hi.s32 dh, %1, %2, ch;\n\tmov.b64 %0, {dl, dh};\n\t}"
            : "=l"(d) : "r"(a[k]), "r"(b), "l"(c[k]));
      }
      c[k] = d;
      asm volatile("" : "+r"(a[k]));
    }
  }
  long long s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k];
  if (s == 0x123456789ll) out[0] = s;
}

}  // namespace
}  // namespace ccg

using namespace ccg;

#define RATE_CUDA(call)                                                  \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) {                                             \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));     \
      return CCG_ERR_CUDA;                                               \
    }                                                                    \
  } while (0)

extern "C" {

ccg_status ccg_pipe_rate(ccg_handle* h, int pipe, double* gops) {
  if (!h || !gops || pipe < 0 || pipe > 4) {
    set_error("ccg_pipe_rate: bad handle, pipe or output pointer");
    return CCG_ERR_INVALID;
  }
  // fewer iterations on the slow FP64 pipe: each timed launch runs ~10 ms
  const int iters = pipe == 0 ? 4096 : 65536;
  const int blocks = h->num_sms * 8, threads = 256;
  void* buf = nullptr;
  RATE_CUDA(cudaMallocAsync(&buf, 512, h->stream));
  std::vector<double> init(32, 1.0000001);
  RATE_CUDA(cudaMemcpyAsync(buf, init.data(), 256, cudaMemcpyHostToDevice, h->stream));
  if (pipe == 1) {
    std::vector<float> f(32, 1.0000001f);
    RATE_CUDA(cudaMemcpyAsync(buf, f.data(), 128, cudaMemcpyHostToDevice, h->stream));
  } else if (pipe >= 2) {
    std::vector<int> v(32);
    for (int k = 0; k < 32; ++k) v[k] = 7 * k + 3;
    RATE_CUDA(cudaMemcpyAsync(buf, v.data(), 128, cudaMemcpyHostToDevice, h->stream));
  }
  auto launch = [&]() {
    char* p = static_cast<char*>(buf);
    if (pipe == 0) rate_dfma<<<blocks, threads, 0, h->stream>>>((const double*)p, (double*)(p + 256), iters);
    else if (pipe == 1) rate_ffma<<<blocks, threads, 0, h->stream>>>((const float*)p, (float*)(p + 256), iters);
    else if (pipe == 2) rate_imad_wide<<<blocks, threads, 0, h->stream>>>((const int*)p, (long long*)(p + 256), iters);
    else if (pipe == 3) rate_mad_ptx<0><<<blocks, threads, 0, h->stream>>>((const int*)p, (long long*)(p + 256), iters);
    else rate_mad_ptx<1><<<blocks, threads, 0, h->stream>>>((const int*)p, (long long*)(p + 256), iters);
  };
  cudaEvent_t e0, e1;
  RATE_CUDA(cudaEventCreate(&e0));
  RATE_CUDA(cudaEventCreate(&e1));
  launch();  // warm-up
  std::vector<float> ts;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0, h->stream);
    launch();
    cudaEventRecord(e1, h->stream);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    ts.push_back(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(buf, h->stream);
  RATE_CUDA(cudaStreamSynchronize(h->stream));
  RATE_CUDA(cudaGetLastError());
  h->launches += 6;
  std::sort(ts.begin(), ts.end());
  const double ops = (double)blocks * threads * iters * kChains;
  *gops = ops / (ts[2] * 1e-3) / 1e9;
  return CCG_OK;
}

}  // extern "C"
