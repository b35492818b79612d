// The fixed-point digit copy of a complex128 dense operator (fx.cuh): made on
// the first integer-pipe sweep, stream-ordered, freed with the operator.
// Layout of the allocation: n x n int4 digits, 256 bytes of padding, the n row
// exponents, then the flag word that marks a non-finite entry (rowexp[n]) and
// the largest row exponent (rowexp[n + 1]).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "fx.cuh"
#include "internal.h"

namespace ccg {

// Operator digits: one warp per row finds the row's largest exponent, then
// writes the row's digits (ar1, ar0, ai1, ai0) into C (leading dimension n).
// *bad is set when A holds an infinity or NaN; bad[1] receives the largest
// row exponent.
__global__ void __launch_bounds__(kBlock) fx_split_matrix(const double2* __restrict__ A, int64_t lda, int64_t n,
                                                          int4* __restrict__ C, int* __restrict__ rowexp,
                                                          int* __restrict__ bad) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * kWarps;
  for (int64_t row = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); row < n; row += warps) {
    const double2* a = A + row * lda;
    int m = 0;
    for (int64_t j = lane; j < n; j += 32) {
      const double2 v = a[j];
      m = max(m, max(fx_exp(v.x), fx_exp(v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      rowexp[row] = m;
      if (m == 0x7FF) atomicExch(bad, 1);
      atomicMax(bad + 1, m);
    }
    int4* c = C + row * n;
    for (int64_t j = lane; j < n; j += 32) {
      const double2 v = a[j];
      int4 q;
      fx_split(v.x, m, q.x, q.y);
      fx_split(v.y, m, q.z, q.w);
      c[j] = q;
    }
  }
}

bool fx_prepare(ccg_handle* h, const ccg_operator* op_c) {
  ccg_operator* op = const_cast<ccg_operator*>(op_c);
  if (op->kind != CCG_OPK_DENSE || op->dtype != CCG_C128) return false;
  if (op->fx_state != 0) return op->fx_state == 1;
  const int64_t n = op->n;
  const size_t cbytes = (size_t)n * (size_t)n * sizeof(int4);
  cudaStream_t s = h->stream;
  op->fx_stream = s;  // stream-ordered: freeing never synchronises the device
  if (cudaMallocAsync(&op->fx_a, cbytes + 256 + (size_t)n * sizeof(int) + 256, s) != cudaSuccess) {
    cudaGetLastError();
    op->fx_a = nullptr;
    op->fx_state = -1;  // not enough memory for the copy: the FP64 pipe it is
    return false;
  }
  char* base = static_cast<char*>(op->fx_a);
  int* rowexp = reinterpret_cast<int*>(base + cbytes + 256);
  int* bad = reinterpret_cast<int*>(base + cbytes + 256 + (size_t)n * sizeof(int));
  if (cudaMemsetAsync(bad, 0, 2 * sizeof(int), s) != cudaSuccess) { cudaGetLastError(); op->fx_state = -1; return false; }
  const int grid = (int)std::min<int64_t>((n + kWarps - 1) / kWarps, (int64_t)h->num_sms * 8);
  fx_split_matrix<<<grid, kBlock, 0, s>>>(static_cast<const double2*>(op->A), op->lda, n, reinterpret_cast<int4*>(base),
                                          rowexp, bad);
  ++h->launches;
  if (cudaGetLastError() != cudaSuccess) { op->fx_state = -1; return false; }
  // a non-finite entry leaves its flag set on the device: the sweeps read it
  // and take the FP64 pipe (no synchronisation here)
  op->fx_state = 1;
  return true;
}

void fx_free(ccg_operator* op) {
  if (op->fx_a) cudaFreeAsync(op->fx_a, op->fx_stream);
  op->fx_a = nullptr;
  op->fx_state = 0;
}

}  // namespace ccg
