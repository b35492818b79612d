// Reductions of libccg's fused update kernels: per-thread accumulators
// (double, or float-float for complex64 data), the single-pass grid
// reduction of the single-right-hand-side phases, and the helpers of the
// fan-in trees of the batched phases and the GMRES passes.
#pragma once

#include "common.cuh"

namespace ccg {

// Per-thread accumulators of the phase kernels' sums: double for complex128
// data; for complex64 data a float-float pair -- each product formed
// exactly (fma) and added by TwoSum -- which keeps about 44 bits of the sum
// on the FP32 pipe instead of widening every element for the (narrow) FP64
// pipe.  The pair becomes a double once per thread, before the block and
// grid reductions.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ void acc_zero(double& a) { a = 0.0; }
__device__ __forceinline__ void acc_zero(FF& a) { a.hi = a.lo = 0.f; }
__device__ __forceinline__ double acc_value(double a) { return a; }
__device__ __forceinline__ double acc_value(const FF& a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ void acc_add1(double& a) { a += 1.0; }
__device__ __forceinline__ void acc_add1(FF& a) { a.hi += 1.f; }
__device__ __forceinline__ void ff_add_prod(FF& s, float x, float y) {
  const float p = x * y;
  const float e = fmaf(x, y, -p);  // x y = p + e exactly
  const float t = s.hi + p;        // TwoSum(s.hi, p) = t + err exactly
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (p - bp);
  s.hi = t;
  s.lo += err + e;
}
// Sum of two float-float values (TwoSum of the high parts, then a
// renormalising Fast2Sum).
__device__ __forceinline__ FF ff_add(const FF& a, const FF& b) {
  const float s = a.hi + b.hi;
  const float bp = s - a.hi;
  const float e = (a.hi - (s - bp)) + (b.hi - bp);
  const float lo = e + a.lo + b.lo;
  const float hi = s + lo;
  FF r;
  r.hi = hi;
  r.lo = lo - (hi - s);
  return r;
}
// Warp sum of one accumulator, valid in lane 0: double shuffles for double,
// float-float shuffles (no FP64 work) for FF.
__device__ __forceinline__ double warp_acc_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_acc_sum(FF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    FF w;
    w.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
    v = ff_add(v, w);
  }
  return acc_value(v);
}

template <class R> struct AccT { typedef double T; };
template <> struct AccT<float> { typedef FF T; };
template <class R> using acc_t = typename AccT<R>::T;

// ---------------------------------------------------------------------------
// Single-pass grid reduction of NQ doubles per thread.  Each block reduces
// in a fixed tree (warp shuffles, then shared memory), writes its partial to
// `partials`, and the last block to arrive sums the partials in block order.
// The result is deterministic for a given grid.  Returns true, with tot[]
// valid in every thread, only in the last block.  `counter` is left at 0.
// ---------------------------------------------------------------------------
template <int NQ, class A>
__device__ __forceinline__ void block_sum(A (&v)[NQ], double (&out)[NQ]) {
  __shared__ double red[NQ][kWarps];
  __shared__ double res[NQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double s = warp_acc_sum(v[q]);
    if (lane == 0) red[q][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = lane < kWarps ? red[q][lane] : 0.0;
#pragma unroll
      for (int o = kWarps / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) res[q] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NQ; ++q) out[q] = res[q];
  __syncthreads();
}

// The same over a group of `nblocks` blocks (block `bid` of the group) of a
// persistent launch; grid_reduce is the whole grid.
template <int NQ, class A>
__device__ __forceinline__ bool group_reduce(A (&v)[NQ], double* __restrict__ partials, unsigned int* counter,
                                             double (&tot)[NQ], int bid, int nblocks) {
  __shared__ bool is_last;
  double bs[NQ];
  block_sum<NQ>(v, bs);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) partials[bid * NQ + q] = bs[q];
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    is_last = (t == (unsigned int)nblocks - 1u);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double s[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) s[q] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kBlock) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) s[q] += __ldcg(&partials[b * NQ + q]);
  }
  block_sum<NQ>(s, tot);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

template <int NQ, class A>
__device__ __forceinline__ bool grid_reduce(A (&v)[NQ], double* __restrict__ partials,
                                            unsigned int* counter, double (&tot)[NQ]) {
  return group_reduce<NQ>(v, partials, counter, tot, blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y);
}


// Fan-in of the cross-block reduction trees (batched phases, the GMRES
// passes), and the counter words a grid needs (one per group of every
// level).
constexpr int kRedGroup = 8;
static inline size_t counter_words(int grid) {
  size_t w = 0;
  for (int cnt = grid; cnt > 1; cnt = (cnt + kRedGroup - 1) / kRedGroup) w += (cnt + kRedGroup - 1) / kRedGroup;
  return w > 0 ? w : 1;
}

// Workspace pointers a reducing kernel needs.
struct Red {
  double* partials;       // kMaxRedBlocks * kMaxNQ doubles
  unsigned int* counter;  // one word, 0 between kernels
};

}  // namespace ccg
