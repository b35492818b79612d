// Shared device-side pieces of libccg: complex arithmetic on interleaved
// (re, im) storage, streaming loads and the per-solve device state.  The
// reductions of the fused update kernels live in reduce.cuh.
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
  int sweeps;     // persistent solve: operator sweeps it ran
};

// Programmatic dependent launch (the kernel-per-step loop launches its
// kernels with it): pdl_wait blocks until the previous kernel in the stream
// has completed and its memory is visible -- so every kernel calls it before
// reading anything -- and pdl_launch lets the next kernel of the stream start
// launching, its blocks then waiting in their own pdl_wait.  Both are no-ops
// for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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

}  // namespace ccg
