// Shared device-side pieces of libccg: complex arithmetic on interleaved
// (re, im) storage, the per-solve device state, and the single-pass grid
// reduction that every fused update kernel ends with.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ccg {

constexpr int kBlock = 256;          // threads per block of every kernel here
constexpr int kWarps = kBlock / 32;
constexpr int kMaxRedBlocks = 2048;  // upper bound on the grid of a reducing kernel
constexpr int kMaxNQ = 32;           // reduction slots per reducing kernel
constexpr int kMaxEll = 4;           // largest degree l of BiCGstab(l)
constexpr int kMaxBasis = 64;        // largest GMRES restart length

// ---------------------------------------------------------------------------
// Complex storage types and arithmetic.
// ---------------------------------------------------------------------------
template <class R> struct Cx;
template <> struct Cx<double> { typedef double2 T; typedef double4 V; };  // V: 16-byte load unit
template <> struct Cx<float> { typedef float2 T; typedef float4 V; };

template <class R> using cx = typename Cx<R>::T;

__host__ __device__ __forceinline__ double2 mkc(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ float2 mkcf(float r, float i) { return make_float2(r, i); }
template <class R> __host__ __device__ __forceinline__ cx<R> mk(R r, R i);
template <> __host__ __device__ __forceinline__ double2 mk<double>(double r, double i) { return make_double2(r, i); }
template <> __host__ __device__ __forceinline__ float2 mk<float>(float r, float i) { return make_float2(r, i); }

template <class T> __host__ __device__ __forceinline__ T cadd(T a, T b) { T c; c.x = a.x + b.x; c.y = a.y + b.y; return c; }
template <class T> __host__ __device__ __forceinline__ T csub(T a, T b) { T c; c.x = a.x - b.x; c.y = a.y - b.y; return c; }
template <class T> __host__ __device__ __forceinline__ T cmul(T a, T b) {
  T c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
template <class T> __host__ __device__ __forceinline__ T cconj(T a) { a.y = -a.y; return a; }
template <class T, class S> __host__ __device__ __forceinline__ T cscale(S s, T a) { a.x *= s; a.y *= s; return a; }
// acc + a*b and acc + conj(a)*b with four fused multiply-adds
template <class T> __device__ __forceinline__ T cfma(T a, T b, T acc) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
  return acc;
}
template <class T> __device__ __forceinline__ T cfma_conj(T a, T b, T acc) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
  return acc;
}
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double cabs(double2 a) { return hypot(a.x, a.y); }
// a / b in double, scaled by the larger component of b (Smith's method).
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  }
  const double r = b.x / b.y, d = b.y + b.x * r;
  return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
template <class R> __device__ __forceinline__ cx<R> narrow(double2 a);
template <> __device__ __forceinline__ double2 narrow<double>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 narrow<float>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <class T> __device__ __forceinline__ double2 widen(T a) { return make_double2((double)a.x, (double)a.y); }

// Breakdown guard: a divisor of modulus below this is treated as zero.
template <class R> __host__ __device__ __forceinline__ double tiny_guard();
template <> __host__ __device__ __forceinline__ double tiny_guard<double>() { return 1e-300; }
template <> __host__ __device__ __forceinline__ double tiny_guard<float>() { return 1e-37; }

// ---------------------------------------------------------------------------
// Streaming loads: the matrix is read once per sweep, so it bypasses L1
// (keeping the reused vector there).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 ld_stream(const double2* p) {
  double2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld_stream(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ld_stream(const float2* p) {
  float2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}

// ---------------------------------------------------------------------------
// Device state of one solve.  The first fields are the poll record the host
// copies back while the solve runs.
// ---------------------------------------------------------------------------
struct Poll {
  int k;          // completed iterations
  int done;       // 1 once the solve has stopped
  int status;     // CCG_OK / CCG_NOT_CONVERGED / CCG_BREAKDOWN / CCG_ERR_NONFINITE
  int breakdown;  // ccg_breakdown
  double relres;  // last recurrence residual
  double ynorm;
};

struct SolveState {
  Poll poll;
  int maxit;
  int half;       // BiCGSTAB took the half-step exit in this iteration
  int zero_rhs;   // y = 0: the host zeroes x
  int skip_mv;    // the start vector is zero: the first product is skipped (reset by the first phase)
  double tol;
  double snorm;   // BiCGSTAB ||s|| / ||y||
  // complex method scalars
  double2 rho, rho_old, alpha, omega, beta, delta, eps, eta, cp, cq;
  // real method scalars
  double gamma, gamma_prev, theta, theta_prev, xi, rho_n, xi_n, c, qrho;
  // GMRES(m): the solve ends with this cycle; Hessenberg columns of the
  // cycle; ||r|| at the cycle start; norm of the last orthogonalised vector
  int gm_final, gm_cols;
  double gm_beta, gm_eta;
  double tau;     // TFQMR quasi-residual norm
  double2 bl_g[kMaxEll];  // BiCGstab(l) minimal-residual coefficients
  double* hist;   // device residual history, maxit + 1 entries
  double* aux;    // spare device doubles for standalone results
};

// A sweep skips when the solve has stopped, is past a half-step exit, or
// starts from x0 = 0.  skip_rec (timed sweeps only) is set by the first
// thread, so that the sweep's duration is left out of the sweep timing.
__device__ __forceinline__ bool sweep_skipped(const SolveState* st, int* skip_rec) {
  if (st == nullptr || !(st->poll.done || st->half || st->skip_mv)) return false;
  if (skip_rec != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *skip_rec = 1;
  return true;
}

// Status codes mirrored from ccg.h for device code.
enum { ST_OK = 0, ST_NOT_CONVERGED = 1, ST_BREAKDOWN = 2, ST_NONFINITE = -4 };

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

template <int NQ, class A>
__device__ __forceinline__ bool grid_reduce(A (&v)[NQ], double* __restrict__ partials,
                                            unsigned int* counter, double (&tot)[NQ]) {
  __shared__ bool is_last;
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
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
