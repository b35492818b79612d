// Dense complex matrix-vector kernels: the manual's `matvec` (y = A x) and
// `cmatvec` (y = A^H x) for a dense row-major A (Sec. 5), plus the fused
// sweep that forms A p and A^H q from one read of A (both products of one
// QMR iteration, Sec. 2.1).
//
// The matrix streams from HBM once per sweep in 16-byte units (one complex
// double, or two complex floats) through loads that skip L1, so that the
// reused vector stays in L1.  Two shapes:
//   * gemv_n_rows: one warp per row, lanes striding along the row; the row
//     sum is a warp reduction and is written directly (no scratch).
//   * gemv_tile: a block owns a column chunk (each lane E units, strided by
//     32 units so every warp load is 512 contiguous bytes) and a row range.
//     A^H x accumulates per column in registers and leaves one partial per
//     row range; A x (in the fused sweep) leaves one partial per column
//     chunk.  Consumers sum the partials (MvOut::get), which keeps the
//     sweep free of atomics and the sums deterministic.
#pragma once

#include "common.cuh"

namespace ccg {

// 16-byte load unit holding U complex numbers of precision R.
template <class R, int U> struct Unit;
template <> struct Unit<double, 1> {
  typedef double2 L;
  static __device__ __forceinline__ double2 get(const L& v, int) { return v; }
  static __device__ __forceinline__ L zero() { return make_double2(0.0, 0.0); }
};
template <> struct Unit<float, 2> {
  typedef float4 L;
  static __device__ __forceinline__ float2 get(const L& v, int c) {
    return c == 0 ? make_float2(v.x, v.y) : make_float2(v.z, v.w);
  }
  static __device__ __forceinline__ L zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <> struct Unit<float, 1> {
  typedef float2 L;
  static __device__ __forceinline__ float2 get(const L& v, int) { return v; }
  static __device__ __forceinline__ L zero() { return make_float2(0.f, 0.f); }
};

__device__ __forceinline__ double2 ldg_unit(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float4 ldg_unit(const float4* p) { return __ldg(p); }
__device__ __forceinline__ float2 ldg_unit(const float2* p) { return __ldg(p); }

// Vector loads of a sweep.  A kernel launch that only reads the vector
// (KC = false) takes the read-only path; inside a persistent solve the same
// vector is rewritten between sweeps (KC = true), so it is read with plain
// coherent loads, which the group barrier's acquire orders after the writes.
__device__ __forceinline__ double2 ldc_unit(const double2* p) {
  double2 v;
  asm volatile("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ldc_unit(const float4* p) {
  float4 v;
  asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ldc_unit(const float2* p) {
  float2 v;
  asm volatile("ld.global.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
template <bool KC, class L> __device__ __forceinline__ L ldv_unit(const L* p) {
  if constexpr (KC) return ldc_unit(p);
  else return ldg_unit(p);
}

template <class T> __device__ __forceinline__ T warp_csum(T s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_down_sync(0xffffffffu, s.x, o);
    s.y += __shfl_down_sync(0xffffffffu, s.y, o);
  }
  return s;
}

// Result of an operator application: either a plain vector y, or `nparts`
// partial vectors P[part * ld + i] whose sum is y (summed in part order), or
// (both null) the zero vector.
template <class R> struct MvOut {
  const cx<R>* y;
  const cx<R>* P;
  int64_t ld;
  int nparts;
  // The partials are added in order 0, 1, ..., nparts - 1; eight loads are
  // issued before their adds so that the reads overlap.
  __device__ __forceinline__ cx<R> get(int64_t i) const {
    if (P == nullptr) return y != nullptr ? y[i] : mk<R>(0, 0);
    cx<R> s = P[i];
    int q = 1;
    for (; q + 7 < nparts; q += 8) {
      cx<R> v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) v[t] = P[(int64_t)(q + t) * ld + i];
#pragma unroll
      for (int t = 0; t < 8; ++t) s = cadd(s, v[t]);
    }
    for (; q < nparts; ++q) s = cadd(s, P[(int64_t)q * ld + i]);
    return s;
  }
};

// y[i] = (A x)_i with S warps per row, each over a contiguous 1/S of the
// row's columns; the S partial sums meet in shared memory and are added in
// warp order.  A block of kWarps warps takes kWarps / S rows at a time.
// Splitting rows makes 4x more work units than one warp per row, so the
// last wave of blocks is a small fraction of the sweep (one warp per row
// left ~1.7 waves of 8-row blocks at n = 8192, the second one 68% full).
// Requires n % U == 0 and 16-byte aligned rows when U * sizeof(cx<R>) == 16.
template <class R, int U, int S, bool KC>
__device__ __forceinline__ void gemv_rows_body(const cx<R>* __restrict__ A, int64_t lda, int64_t n,
                                               const cx<R>* x, cx<R>* y, int64_t lb, int64_t G) {
  typedef Unit<R, U> Un;
  typedef typename Un::L L;
  static_assert(kWarps % S == 0, "S must divide the warps of a block");
  constexpr int RPB = kWarps / S;  // rows per block pass
  __shared__ cx<R> part[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = warp % S;
  const int64_t nunits = n / U;
  const int64_t u0 = nunits * seg / S, u1 = nunits * (seg + 1) / S;
  const L* xv = reinterpret_cast<const L*>(x);
  const int64_t nrb = (n + RPB - 1) / RPB;
  for (int64_t rb = lb; rb < nrb; rb += G) {
    const int64_t row = rb * RPB + warp / S;
    cx<R> s0 = mk<R>(0, 0), s1 = mk<R>(0, 0);
    if (row < n) {
      const L* a = reinterpret_cast<const L*>(A + row * lda);
      int64_t u = u0 + lane;
      for (; u + 96 < u1; u += 128) {
        const L a0 = ld_stream(a + u), a1 = ld_stream(a + u + 32), a2 = ld_stream(a + u + 64),
                a3 = ld_stream(a + u + 96);
        const L x0 = ldv_unit<KC>(xv + u), x1 = ldv_unit<KC>(xv + u + 32), x2 = ldv_unit<KC>(xv + u + 64),
                x3 = ldv_unit<KC>(xv + u + 96);
#pragma unroll
        for (int c = 0; c < U; ++c) {
          s0 = cfma(Un::get(a0, c), Un::get(x0, c), s0);
          s1 = cfma(Un::get(a1, c), Un::get(x1, c), s1);
          s0 = cfma(Un::get(a2, c), Un::get(x2, c), s0);
          s1 = cfma(Un::get(a3, c), Un::get(x3, c), s1);
        }
      }
      for (; u < u1; u += 32) {
        const L a0 = ld_stream(a + u), x0 = ldv_unit<KC>(xv + u);
#pragma unroll
        for (int c = 0; c < U; ++c) s0 = cfma(Un::get(a0, c), Un::get(x0, c), s0);
      }
    }
    const cx<R> ws = warp_csum(cadd(s0, s1));
    if (S == 1) {
      if (lane == 0 && row < n) y[row] = ws;
    } else {
      if (lane == 0) part[warp] = ws;
      __syncthreads();
      if (seg == 0 && lane == 0 && row < n) {
        cx<R> t = part[warp];
#pragma unroll
        for (int q = 1; q < S; ++q) t = cadd(t, part[warp + q]);
        y[row] = t;
      }
      __syncthreads();
    }
  }
}

template <class R, int U, int S = 1>
__global__ void __launch_bounds__(kBlock) gemv_n_rows(const cx<R>* __restrict__ A, int64_t lda, int64_t n,
                                                      const cx<R>* __restrict__ x, cx<R>* __restrict__ y,
                                                      const SolveState* __restrict__ st, int* skip_rec = nullptr) {
  pdl_wait();
  if (sweep_skipped(st, skip_rec)) {
    pdl_launch();
    return;
  }
  gemv_rows_body<R, U, S, false>(A, lda, n, x, y, blockIdx.x, gridDim.x);
  pdl_launch();
}

// Column-tiled sweep.  grid = (column chunks, row ranges).  With Y1 it
// writes P1[chunk * n + row] = sum over the chunk's columns of A[row, c] x1[c];
// with Y2 it writes P2[range * n + col] = sum over the range's rows of
// conj(A[row, col]) x2[row].
// x2 values of a row: read-only path in a plain launch, coherent loads in a
// persistent solve (see ldv_unit).
template <bool KC, class T> __device__ __forceinline__ T ldv_elem(const T* p) {
  if constexpr (KC) {
    return ldc_unit(p);
  } else {
    return __ldg(p);
  }
}

// One tile: column chunk `chunk` (32 E units) and row range `range`.  KC as
// in gemv_rows_body.
// Shared memory of a tile's column sums: kWarps x 32 E U complex values.
template <class R, int U, int E> constexpr int tile_smem_elems() { return kWarps * 32 * E * U; }

template <class R, int U, int E, bool Y1, bool Y2, bool KC = false>
__device__ __forceinline__ void gemv_tile_body(const cx<R>* __restrict__ A, int64_t lda, int64_t n,
                                               int64_t rows_per_range, const cx<R>* x1, const cx<R>* x2,
                                               cx<R>* P1, cx<R>* P2, int64_t chunk, int64_t range,
                                               cx<R>* smem_ext = nullptr) {
  typedef Unit<R, U> Un;
  typedef typename Un::L L;
  constexpr int CBU = 32 * E;  // units per column chunk
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nunits = n / U;
  const int64_t unit0 = chunk * CBU;
  const int64_t r0 = range * rows_per_range;
  const int64_t r1 = r0 + rows_per_range < n ? r0 + rows_per_range : n;

  L xl[E];
  if (Y1) {
    const L* xv = reinterpret_cast<const L*>(x1);
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int64_t u = unit0 + lane + 32 * j;
      xl[j] = u < nunits ? ldv_unit<KC>(xv + u) : Un::zero();
    }
  }
  cx<R> acc[E][U];
#pragma unroll
  for (int j = 0; j < E; ++j)
#pragma unroll
    for (int c = 0; c < U; ++c) acc[j][c] = mk<R>(0, 0);

  if constexpr (Y1) {
    // A x1 (and A^H x2): one row per iteration per warp
    for (int64_t r = r0 + warp; r < r1; r += kWarps) {
      const L* a = reinterpret_cast<const L*>(A + r * lda);
      L av[E];
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int64_t u = unit0 + lane + 32 * j;
        av[j] = u < nunits ? ld_stream(a + u) : Un::zero();
      }
      if (Y2) {
        const cx<R> xr = ldv_elem<KC>(x2 + r);
#pragma unroll
        for (int j = 0; j < E; ++j)
#pragma unroll
          for (int c = 0; c < U; ++c) acc[j][c] = cfma_conj(Un::get(av[j], c), xr, acc[j][c]);
      }
      cx<R> s = mk<R>(0, 0);
#pragma unroll
      for (int j = 0; j < E; ++j)
#pragma unroll
        for (int c = 0; c < U; ++c) s = cfma(Un::get(av[j], c), Un::get(xl[j], c), s);
      s = warp_csum(s);
      if (lane == 0) P1[chunk * n + r] = s;
    }
  } else if constexpr (sizeof(R) == 8) {
    // A^H x2 alone, complex128: bound by the FP64 pipe, one row per iteration
    for (int64_t r = r0 + warp; r < r1; r += kWarps) {
      const L* a = reinterpret_cast<const L*>(A + r * lda);
      L av[E];
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int64_t u = unit0 + lane + 32 * j;
        av[j] = u < nunits ? ld_stream(a + u) : Un::zero();
      }
      const cx<R> xr = ldv_elem<KC>(x2 + r);
#pragma unroll
      for (int j = 0; j < E; ++j)
#pragma unroll
        for (int c = 0; c < U; ++c) acc[j][c] = cfma_conj(Un::get(av[j], c), xr, acc[j][c]);
    }
  } else {
    // A^H x2 alone, complex64: the warp's rows r0 + warp + kWarps t take their
    // x2 values 32 at a time in one coalesced load, passed out by shuffles,
    // and two rows are streamed per iteration (2 E loads per lane in flight):
    // 0.115 -> 0.097 ms at n = 8192.  (With Y1 the extra registers would cut
    // the resident blocks and cost more than they save.)
    const int64_t rw = r0 + warp;
    const int64_t nrw = rw < r1 ? (r1 - rw + kWarps - 1) / kWarps : 0;
    for (int64_t t0 = 0; t0 < nrw; t0 += 32) {
      cx<R> xlane = mk<R>(0, 0);
      if (t0 + lane < nrw) xlane = ldv_elem<KC>(x2 + rw + kWarps * (t0 + lane));
      const int cnt = (int)(nrw - t0 < 32 ? nrw - t0 : 32);
      int t = 0;
      for (; t + 1 < cnt; t += 2) {
        const int64_t ra = rw + kWarps * (t0 + t), rb = ra + kWarps;
        const L* a = reinterpret_cast<const L*>(A + ra * lda);
        const L* b = reinterpret_cast<const L*>(A + rb * lda);
        L av[E], bv[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const int64_t u = unit0 + lane + 32 * j;
          av[j] = u < nunits ? ld_stream(a + u) : Un::zero();
          bv[j] = u < nunits ? ld_stream(b + u) : Un::zero();
        }
        const cx<R> xa = mk<R>(__shfl_sync(0xffffffffu, xlane.x, t), __shfl_sync(0xffffffffu, xlane.y, t));
        const cx<R> xb = mk<R>(__shfl_sync(0xffffffffu, xlane.x, t + 1), __shfl_sync(0xffffffffu, xlane.y, t + 1));
#pragma unroll
        for (int j = 0; j < E; ++j)
#pragma unroll
          for (int c = 0; c < U; ++c) {
            acc[j][c] = cfma_conj(Un::get(av[j], c), xa, acc[j][c]);
            acc[j][c] = cfma_conj(Un::get(bv[j], c), xb, acc[j][c]);
          }
      }
      if (t < cnt) {
        const int64_t ra = rw + kWarps * (t0 + t);
        const L* a = reinterpret_cast<const L*>(A + ra * lda);
        L av[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const int64_t u = unit0 + lane + 32 * j;
          av[j] = u < nunits ? ld_stream(a + u) : Un::zero();
        }
        const cx<R> xa = mk<R>(__shfl_sync(0xffffffffu, xlane.x, t), __shfl_sync(0xffffffffu, xlane.y, t));
#pragma unroll
        for (int j = 0; j < E; ++j)
#pragma unroll
          for (int c = 0; c < U; ++c) acc[j][c] = cfma_conj(Un::get(av[j], c), xa, acc[j][c]);
      }
    }
  }
  if (Y2) {
    // a persistent launch passes one buffer for all its tile shapes
    cx<R>* sm;
    if constexpr (KC) {
      sm = smem_ext;
    } else {
      __shared__ cx<R> sm_own[kWarps * CBU * U];
      sm = sm_own;
    }
#pragma unroll
    for (int j = 0; j < E; ++j)
#pragma unroll
      for (int c = 0; c < U; ++c) sm[warp * CBU * U + (lane + 32 * j) * U + c] = acc[j][c];
    __syncthreads();
    for (int t = threadIdx.x; t < CBU * U; t += kBlock) {
      const int64_t col = unit0 * U + t;
      if (col < n) {
        cx<R> s = sm[t];
#pragma unroll
        for (int w = 1; w < kWarps; ++w) s = cadd(s, sm[w * CBU * U + t]);
        P2[range * n + col] = s;
      }
    }
    if (KC) __syncthreads();   // a persistent block's next tile reuses sm
  }
}

// Entry points: with Y1 (A x1, optionally with A^H x2) the compiler's own
// register choice keeps 4 blocks per SM at complex64; A^H x alone in
// complex64 is held to 3 blocks per SM.
template <class R, int U, int E, bool Y1, bool Y2>
__global__ void __launch_bounds__(kBlock) gemv_tile(const cx<R>* __restrict__ A, int64_t lda, int64_t n,
                                                    int64_t rows_per_range, const cx<R>* __restrict__ x1,
                                                    const cx<R>* __restrict__ x2, cx<R>* __restrict__ P1,
                                                    cx<R>* __restrict__ P2, const SolveState* __restrict__ st,
                                                    int* skip_rec = nullptr) {
  static_assert(Y1, "A^H x alone runs in gemv_tile_h");
  pdl_wait();
  if (sweep_skipped(st, skip_rec)) {
    pdl_launch();
    return;
  }
  gemv_tile_body<R, U, E, Y1, Y2>(A, lda, n, rows_per_range, x1, x2, P1, P2, blockIdx.x, blockIdx.y);
  pdl_launch();
}
template <class R, int U, int E>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 3 : 1)
    gemv_tile_h(const cx<R>* __restrict__ A, int64_t lda, int64_t n, int64_t rows_per_range,
                const cx<R>* __restrict__ x2, cx<R>* __restrict__ P2, const SolveState* __restrict__ st,
                int* skip_rec = nullptr) {
  pdl_wait();
  if (sweep_skipped(st, skip_rec)) {
    pdl_launch();
    return;
  }
  gemv_tile_body<R, U, E, false, true>(A, lda, n, rows_per_range, nullptr, x2, nullptr, P2, blockIdx.x, blockIdx.y);
  pdl_launch();
}

}  // namespace ccg
