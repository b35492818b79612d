// Complex128 y = A x on the integer pipe instead of GB300's narrow FP64 pipe.
//
// A complex128 row sweep needs 4 DFMA per 16-byte element, and GB300 retires
// 2 DFMA per SM clock (measured: 1.25 TFLOP/s), so the FP64 pipe caps the
// sweep at about 2.3 TB/s, a third of HBM.  Here each row of A and the vector
// x are written in fixed point with 53 significant bits (the row's, resp.
// the vector's, largest binary exponent as the scale; the error-free
// splitting of Ozaki et al. carried to integers, as in the block products of
// tc_ozaki.cu), each 53-bit integer is cut into two balanced 26-bit digits,
// and a product a x is formed exactly from the digit products
// a1 x1 2^52 + (a1 x0 + a0 x1) 2^26 by 64-bit integer multiply-adds
// (IMAD.WIDE, ~60 per SM clock); only a0 x0 < 2^50 units is left out.  The
// row sums are exact in int64 and converted to double every 256 elements.
//
// Accuracy per output: |error| <= 2.5 n 2^(Fa + Fx - 52) where 2^Fa > max|a_ij|
// over the row and 2^Fx > max|x_j| -- the bound of an FP64 GEMV relative to
// the row's and vector's largest entries (an FP64 GEMV's is relative to
// sum |a_ij||x_j|); entries far below their row's largest keep fewer bits.
//
// The digits of A are made once per operator (16 bytes per element, as A
// itself) and read in place of A; those of x once per sweep.  A matrix with
// a non-finite entry (flagged on the device when the digits are made), or a
// vector with one, takes the FP64-pipe sweep.
#pragma once

#include "common.cuh"
#include "gemv.cuh"

namespace ccg {

// Fixed-point digits (d1, d0) of v with d1 2^26 + d0 = round(v 2^(52 - F))
// where F = max(emax, 1) - 1022 is the scale of the row or vector whose
// largest biased exponent is emax; |d1| <= 2^26, -2^25 <= d0 < 2^25.
__device__ __forceinline__ void fx_split(double v, int emax, int& d1, int& d0) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = (unsigned)(b >> 32);
  const int E = (hi >> 20) & 0x7FF;
  const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | ((unsigned long long)(E != 0) << 52);
  int d = max(emax, 1) - max(E, 1) + 1;  // >= 1 since emax >= E
  d = min(d, 63);                         // M < 2^53: any d >= 54 rounds to 0
  long long r = (long long)((M + (1ull << (d - 1))) >> d);
  if (hi >> 31) r = -r;
  const long long a1 = (r + (1ll << 25)) >> 26;
  d1 = (int)a1;
  d0 = (int)(r - (a1 << 26));
}

__device__ __forceinline__ int fx_exp(double v) { return (int)((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FF; }

// A^H x sums down the columns of A, whose rows have different scales, so the
// vector of that sweep is first scaled row by row: x'_r = x_r 2^(F_r - Fm),
// Fm the largest row scale (exact but for subnormal results), and every
// product conj(a_rc) x_r then has the one scale 2^(Fm + Fx' - 104).
__device__ __forceinline__ double2 fx_row_scaled(double2 v, int er, int fm) {
  const int sh = max(er, 1) - fm;  // <= 0
  return make_double2(ldexp(v.x, sh), ldexp(v.y, sh));
}

// Vector digits for one sweep (one block): the largest exponent of x (of x'
// with ROWS: rowexp as the operator's, rowexp[n + 1] its largest row
// exponent), then the digits (xr1, xr0, xi1, xi0).  meta[0] = the exponent,
// meta[1] = 1 when x holds an infinity or NaN.
template <int THREADS, bool ROWS>
__device__ __forceinline__ void fx_split_block(const double2* __restrict__ x, int64_t n, int4* __restrict__ xd,
                                               int* __restrict__ meta, const int* __restrict__ rowexp) {
  __shared__ int wm[THREADS / 32];
  const int fm = ROWS ? max(rowexp[n + 1], 1) : 0;
  int m = 0;
  for (int64_t j = threadIdx.x; j < n; j += THREADS) {
    double2 v = x[j];
    if (ROWS) v = fx_row_scaled(v, rowexp[j], fm);
    m = max(m, max(fx_exp(v.x), fx_exp(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0;
#pragma unroll
  for (int w = 0; w < THREADS / 32; ++w) m = max(m, wm[w]);
  if (threadIdx.x == 0) {
    meta[0] = m;
    meta[1] = m == 0x7FF ? 1 : 0;
  }
  for (int64_t j = threadIdx.x; j < n; j += THREADS) {
    double2 v = x[j];
    if (ROWS) v = fx_row_scaled(v, rowexp[j], fm);
    int4 q;
    fx_split(v.x, m, q.x, q.y);
    fx_split(v.y, m, q.z, q.w);
    xd[j] = q;
  }
}

template <int THREADS, bool ROWS>
__global__ void __launch_bounds__(THREADS) fx_split_vector(const double2* __restrict__ x, int64_t n,
                                                           int4* __restrict__ xd, int* __restrict__ meta,
                                                           const SolveState* __restrict__ st,
                                                           const int* __restrict__ rowexp) {
  pdl_wait();
  pdl_launch();
  if (sweep_skipped(st, nullptr)) return;
  fx_split_block<THREADS, ROWS>(x, n, xd, meta, rowexp);
}

// Exact complex digit products into int64: re += ar xr - ai xi,
// im += ar xi + ai xr, high digit products (x 2^52) apart from the middle
// ones (x 2^26).
struct FxAcc {
  long long hre, mre, him, mim;
  __device__ __forceinline__ void zero() { hre = mre = him = mim = 0; }
  __device__ __forceinline__ void mac(const int4 a, const int4 x) {
    const int nai1 = -a.z, nai0 = -a.w;
    hre += (long long)a.x * x.x;
    hre += (long long)nai1 * x.z;
    mre += (long long)a.x * x.y;
    mre += (long long)a.y * x.x;
    mre += (long long)nai1 * x.w;
    mre += (long long)nai0 * x.z;
    him += (long long)a.x * x.z;
    him += (long long)a.z * x.x;
    mim += (long long)a.x * x.w;
    mim += (long long)a.y * x.z;
    mim += (long long)a.z * x.y;
    mim += (long long)a.w * x.x;
  }
  // the sums so far in units of 2^(Fa + Fx - 78), exactly up to the rounding
  // of the int64 -> double conversions
  __device__ __forceinline__ void flush(double& re, double& im) {
    re += (double)hre * 67108864.0 + (double)mre;
    im += (double)him * 67108864.0 + (double)mim;
    zero();
  }
};

// The same for conj(a) x: re += ar xr + ai xi, im += ar xi - ai xr.
struct FxAccH {
  long long hre, mre, him, mim;
  __device__ __forceinline__ void zero() { hre = mre = him = mim = 0; }
  __device__ __forceinline__ void mac(const int4 a, const int4 x) {
    const int nai1 = -a.z, nai0 = -a.w;
    hre += (long long)a.x * x.x;
    hre += (long long)a.z * x.z;
    mre += (long long)a.x * x.y;
    mre += (long long)a.y * x.x;
    mre += (long long)a.z * x.w;
    mre += (long long)a.w * x.z;
    him += (long long)a.x * x.z;
    him += (long long)nai1 * x.x;
    mim += (long long)a.x * x.w;
    mim += (long long)a.y * x.z;
    mim += (long long)nai1 * x.y;
    mim += (long long)nai0 * x.x;
  }
  __device__ __forceinline__ void flush(double& re, double& im) {
    re += (double)hre * 67108864.0 + (double)mre;
    im += (double)him * 67108864.0 + (double)mim;
    zero();
  }
};

__device__ __forceinline__ int4 ld_stream_i4(const int4* p) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ int4 ldc_i4(const int4* p) {
  int4 v;
  asm volatile("ld.global.v4.s32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}

// y = A x from the digits: S warps per row as in gemv_rows_body, 8 loads in
// flight per lane, int64 sums flushed to double every 256 elements.  The
// sweep waits on its loads, not on the integer pipe: on the GB300 two warps
// per row with 8 loads in flight ran n = 8192 in 0.19 ms where four warps
// with 4 took 0.23 ms.  With
// meta[1] set (x not finite) the rows are summed from A on the FP64 pipe.
// KC as in gemv_rows_body (the digits of x are rewritten between sweeps of a
// persistent solve).
template <int S, bool KC>
__device__ __forceinline__ void gemv_fx_rows_body(const double2* __restrict__ A, int64_t lda, const int4* __restrict__ C,
                                                  const int* __restrict__ rowexp, int64_t n, const double2* x,
                                                  const int4* xd, int xexp, bool xbad, double2* y, int64_t lb,
                                                  int64_t G) {
  constexpr int RPB = kWarps / S;
  __shared__ double2 part[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = warp % S;
  const int64_t u0 = n * seg / S, u1 = n * (seg + 1) / S;
  const int64_t nrb = (n + RPB - 1) / RPB;
  for (int64_t rb = lb; rb < nrb; rb += G) {
    const int64_t row = rb * RPB + warp / S;
    double sre = 0.0, sim = 0.0;
    int er = 0;
    if (row < n) {
      if (xbad) {
        const double2* a = A + row * lda;
        double2 s0 = make_double2(0.0, 0.0);
        for (int64_t u = u0 + lane; u < u1; u += 32) s0 = cfma(ld_stream(a + u), ldv_unit<KC>(x + u), s0);
        sre = s0.x;
        sim = s0.y;
      } else {
        er = rowexp[row];
        const int4* c = C + row * n;
        int64_t u = u0 + lane;
        FxAcc acc;
        while (u < u1) {
          acc.zero();
          const int64_t uend = u + 256 * 32 < u1 ? u + 256 * 32 : u1;
          for (; u + 224 < uend; u += 256) {
            int4 q[8], xv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) q[k] = ld_stream_i4(c + u + 32 * k);
#pragma unroll
            for (int k = 0; k < 8; ++k) xv[k] = KC ? ldc_i4(xd + u + 32 * k) : __ldg(xd + u + 32 * k);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc.mac(q[k], xv[k]);
          }
          for (; u < uend; u += 32) {
            const int4 xv = KC ? ldc_i4(xd + u) : __ldg(xd + u);
            acc.mac(ld_stream_i4(c + u), xv);
          }
          acc.flush(sre, sim);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sre += __shfl_down_sync(0xffffffffu, sre, o);
      sim += __shfl_down_sync(0xffffffffu, sim, o);
    }
    if (lane == 0) part[warp] = make_double2(sre, sim);
    __syncthreads();
    if (seg == 0 && lane == 0 && row < n) {
      double2 t = part[warp];
#pragma unroll
      for (int q = 1; q < S; ++q) t = cadd(t, part[warp + q]);
      if (!xbad) {
        const int e = max(er, 1) + max(xexp, 1) - 2122;  // units 2^(Fa + Fx - 78)
        t = make_double2(ldexp(t.x, e), ldexp(t.y, e));
      }
      y[row] = t;
    }
    __syncthreads();
  }
}

// rowexp[n] (the word after the row exponents) marks a non-finite entry of A.
template <int S>
__global__ void __launch_bounds__(kBlock) gemv_fx_rows(const double2* __restrict__ A, int64_t lda,
                                                       const int4* __restrict__ C, const int* __restrict__ rowexp,
                                                       int64_t n, const double2* __restrict__ x,
                                                       const int4* __restrict__ xd, const int* __restrict__ meta,
                                                       double2* __restrict__ y, const SolveState* __restrict__ st,
                                                       int* skip_rec = nullptr) {
  pdl_wait();
  if (sweep_skipped(st, skip_rec)) {
    pdl_launch();
    return;
  }
  gemv_fx_rows_body<S, false>(A, lda, C, rowexp, n, x, xd, meta[0], meta[1] != 0 || rowexp[n] != 0, y, blockIdx.x,
                              gridDim.x);
  pdl_launch();
}

// A^H x on the integer pipe over the tiles of gemv_tile_body (column chunk
// of 128 columns, a lane per 4 columns, row range `range` of rows_per_range
// rows; the same partial-sum output).  xd2 holds the digits of the
// row-scaled x' (exponent xexp2; rowexp[n + 1] is the operator's largest row
// exponent).  Each column accumulates exactly in int64 per warp, two rows
// per iteration (8 loads of 16 bytes in flight per lane), converted to
// double every 256 rows.  KC as in gemv_rows_body; smem_ext as in
// gemv_tile_body.  (A fused form that also formed A x1 from the same read
// reduced each row's chunk sum across the warp and ran at 0.58 ms at
// n = 8192, slower than this sweep and the row sweep run one after the
// other, 0.26 + 0.20 ms: the complex128 A p + A^H q uses the two.)
template <bool KC>
__device__ __forceinline__ void gemv_fx_tile_body(const int4* __restrict__ C, const int* __restrict__ rowexp,
                                                  int64_t n, int64_t rows_per_range, const int4* xd2, int xexp2,
                                                  double2* P2, int64_t chunk, int64_t range,
                                                  double2* smem_ext = nullptr) {
  constexpr int E = 4, CBU = 32 * E;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t col0 = chunk * CBU;
  const int64_t r0 = range * rows_per_range;
  const int64_t r1 = r0 + rows_per_range < n ? r0 + rows_per_range : n;
  const int fm = max(rowexp[n + 1], 1);
  FxAccH acc[E];
  double dre[E], dim[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    acc[j].zero();
    dre[j] = 0.0;
    dim[j] = 0.0;
  }
  int cnt = 0;
  int64_t r = r0 + warp;
  for (; r + kWarps < r1; r += 2 * kWarps) {
    const int4* ca = C + r * n;
    const int4* cb = ca + kWarps * n;
    int4 av[E], bv[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int64_t u = col0 + lane + 32 * j;
      av[j] = u < n ? ld_stream_i4(ca + u) : make_int4(0, 0, 0, 0);
      bv[j] = u < n ? ld_stream_i4(cb + u) : make_int4(0, 0, 0, 0);
    }
    const int4 xa = KC ? ldc_i4(xd2 + r) : __ldg(xd2 + r);
    const int4 xb = KC ? ldc_i4(xd2 + r + kWarps) : __ldg(xd2 + r + kWarps);
#pragma unroll
    for (int j = 0; j < E; ++j) {
      acc[j].mac(av[j], xa);
      acc[j].mac(bv[j], xb);
    }
    if ((cnt += 2) >= 256) {
#pragma unroll
      for (int j = 0; j < E; ++j) acc[j].flush(dre[j], dim[j]);
      cnt = 0;
    }
  }
  for (; r < r1; r += kWarps) {
    const int4* c = C + r * n;
    int4 av[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int64_t u = col0 + lane + 32 * j;
      av[j] = u < n ? ld_stream_i4(c + u) : make_int4(0, 0, 0, 0);
    }
    const int4 xr = KC ? ldc_i4(xd2 + r) : __ldg(xd2 + r);
#pragma unroll
    for (int j = 0; j < E; ++j) acc[j].mac(av[j], xr);
    if (++cnt >= 256) {
#pragma unroll
      for (int j = 0; j < E; ++j) acc[j].flush(dre[j], dim[j]);
      cnt = 0;
    }
  }
#pragma unroll
  for (int j = 0; j < E; ++j) acc[j].flush(dre[j], dim[j]);
  double2* sm;
  if constexpr (KC) {
    sm = smem_ext;
  } else {
    __shared__ double2 sm_own[kWarps * CBU];
    sm = sm_own;
  }
#pragma unroll
  for (int j = 0; j < E; ++j) sm[warp * CBU + lane + 32 * j] = make_double2(dre[j], dim[j]);
  __syncthreads();
  const int e2 = fm + max(xexp2, 1) - 2122;  // units 2^(Fm + Fx' - 78)
  for (int t = threadIdx.x; t < CBU; t += kBlock) {
    const int64_t col = col0 + t;
    if (col < n) {
      double2 v = sm[t];
#pragma unroll
      for (int w = 1; w < kWarps; ++w) v = cadd(v, sm[w * CBU + t]);
      P2[range * n + col] = make_double2(ldexp(v.x, e2), ldexp(v.y, e2));
    }
  }
  if (KC) __syncthreads();  // a persistent block's next tile reuses sm
}

// The same sweep with the digit rows staged through shared memory: each
// warp keeps kFxStages rows of its tile in flight with cp.async (16-byte
// copies that bypass L1), so the loads no longer wait on registers: the
// register-held form (gemv_fx_tile_body) stopped at 2 blocks per SM with
// 8 loads in flight per lane.  A lane copies and later reads only its own 4
// columns of each row, so no synchronisation within the warp is needed.
// Rows, flush points and the final sums are those of gemv_fx_tile_body, so
// the results are bitwise the same.  smem: kFxStages x 128 int4 per warp.
constexpr int kFxStages = 4;
constexpr size_t kFxTileSmem = (size_t)kWarps * kFxStages * 128 * sizeof(int4);

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void gemv_fx_tile_staged(const int4* __restrict__ C, const int* __restrict__ rowexp,
                                                    int64_t n, int64_t rows_per_range, const int4* __restrict__ xd2,
                                                    int xexp2, double2* P2, int64_t chunk, int64_t range,
                                                    int4* stage) {
  constexpr int E = 4, CBU = 32 * E;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t col0 = chunk * CBU;
  const int64_t r0 = range * rows_per_range;
  const int64_t r1 = r0 + rows_per_range < n ? r0 + rows_per_range : n;
  const int fm = max(rowexp[n + 1], 1);
  int4* ws = stage + (size_t)warp * kFxStages * CBU;
  // row k of this warp (r0 + warp + k kWarps) into ring slot k mod kFxStages;
  // columns beyond n are filled with zeros (source address kept in the row)
  auto issue = [&](int64_t k) {
    const int64_t r = r0 + warp + k * kWarps;
    if (r < r1) {
      const int4* src = C + r * n;
      int4* dst = ws + (int)(k % kFxStages) * CBU;
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int64_t u = col0 + lane + 32 * j;
        cp_async16(dst + lane + 32 * j, src + (u < n ? u : 0), u < n ? 16 : 0);
      }
    }
    cp_async_commit();
  };
  FxAccH acc[E];
  double dre[E], dim[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    acc[j].zero();
    dre[j] = 0.0;
    dim[j] = 0.0;
  }
#pragma unroll
  for (int k = 0; k < kFxStages - 1; ++k) issue(k);
  int cnt = 0;
  int64_t k = 0;
  for (int64_t r = r0 + warp; r < r1; r += kWarps, ++k) {
    issue(k + kFxStages - 1);
    cp_async_wait<kFxStages - 1>();
    const int4* row = ws + (int)(k % kFxStages) * CBU;
    const int4 xr = __ldg(xd2 + r);
#pragma unroll
    for (int j = 0; j < E; ++j) acc[j].mac(row[lane + 32 * j], xr);
    if (++cnt >= 256) {
#pragma unroll
      for (int j = 0; j < E; ++j) acc[j].flush(dre[j], dim[j]);
      cnt = 0;
    }
  }
  cp_async_wait<0>();
#pragma unroll
  for (int j = 0; j < E; ++j) acc[j].flush(dre[j], dim[j]);
  // the warps' column sums, each through its own warp's ring (16-byte
  // slots, like the int4 rows)
  double2* sm = reinterpret_cast<double2*>(stage);
  constexpr int WS = kFxStages * CBU;
#pragma unroll
  for (int j = 0; j < E; ++j) sm[warp * WS + lane + 32 * j] = make_double2(dre[j], dim[j]);
  __syncthreads();
  const int e2 = fm + max(xexp2, 1) - 2122;  // units 2^(Fm + Fx' - 78)
  for (int t = threadIdx.x; t < CBU; t += kBlock) {
    const int64_t col = col0 + t;
    if (col < n) {
      double2 v = sm[t];
#pragma unroll
      for (int w = 1; w < kWarps; ++w) v = cadd(v, sm[w * WS + t]);
      P2[range * n + col] = make_double2(ldexp(v.x, e2), ldexp(v.y, e2));
    }
  }
}

// Entry point of the integer A^H x sweep (kFxTileSmem bytes of dynamic
// shared memory).  With a non-finite entry in A (rowexp[n]) or in the vector
// (meta[1]) the tile is summed from A on the FP64 pipe instead.
static __global__ void __launch_bounds__(kBlock, 3) gemv_fx_tile_h(const double2* __restrict__ A, int64_t lda,
                                                                const int4* __restrict__ C,
                                                                const int* __restrict__ rowexp, int64_t n,
                                                                int64_t rows_per_range,
                                                                const double2* __restrict__ x,
                                                                const int4* __restrict__ xd,
                                                                const int* __restrict__ meta, double2* __restrict__ P2,
                                                                const SolveState* __restrict__ st,
                                                                int* skip_rec = nullptr) {
  extern __shared__ int4 fx_stage[];
  pdl_wait();
  if (sweep_skipped(st, skip_rec)) {
    pdl_launch();
    return;
  }
  if (rowexp[n] != 0 || meta[1] != 0) {
    gemv_tile_body<double, 1, 4, false, true, true>(A, lda, n, rows_per_range, nullptr, x, nullptr, P2, blockIdx.x,
                                                    blockIdx.y, reinterpret_cast<double2*>(fx_stage));
  } else {
    gemv_fx_tile_staged(C, rowexp, n, rows_per_range, xd, meta[0], P2, blockIdx.x, blockIdx.y, fx_stage);
  }
  pdl_launch();
}

}  // namespace ccg
