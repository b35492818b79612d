// Multi-right-hand-side dense products on CUDA cores: C = A B for complex A
// (n x n, row-major, leading dimension lda) and blocks B, C of k right-hand
// sides stored row-major (row i holds the k values of unknown i, leading
// dimension k), in complex128 or complex64.
//
// A block of 16 x 16 threads computes a (16 TM) x (16 TN) tile of C; each
// thread owns a TM x TN sub-tile of complex accumulators in registers.  K
// advances 8 complex values at a time through shared memory (A transposed so
// that a thread's rows are one broadcast-friendly load).  complex128 is bound
// by the FP64 pipe (4 DFMA per complex multiply-add); complex64 by the FP32
// pipe.
#pragma once

#include "common.cuh"

namespace ccg {

// Tile shape per precision: complex64 64 x 64 (4 x 4 per thread, FP32 pipe
// and shared-memory bandwidth balanced); complex128 32 x 32 (2 x 2 per
// thread): the FP64 pipe is so much slower than shared memory that smaller
// tiles cost nothing, and 4x more blocks fill the 152 SMs in ~14 waves
// instead of ~3.4 (a partial last wave alone cost 16%).
template <class R> struct GemmTile;
template <> struct GemmTile<float> { static constexpr int TM = 4, TN = 4; };
template <> struct GemmTile<double> { static constexpr int TM = 2, TN = 2; };
constexpr int kGemmBK = 8;
template <class R> constexpr int gemm_bm() { return 16 * GemmTile<R>::TM; }
template <class R> constexpr int gemm_bn() { return 16 * GemmTile<R>::TN; }

template <class R>
__global__ void __launch_bounds__(kBlock) cgemm_rows(const cx<R>* __restrict__ A, int64_t lda,
                                                     const cx<R>* __restrict__ B, cx<R>* __restrict__ C, int64_t n,
                                                     int k, const int* __restrict__ skip, int* skip_rec = nullptr) {
  constexpr int TM = GemmTile<R>::TM, TN = GemmTile<R>::TN;
  constexpr int BM = 16 * TM, BN = 16 * TN;
  constexpr int A_PER = BM * kGemmBK / kBlock, B_PER = kGemmBK * BN / kBlock;
  if (skip != nullptr && *skip) {  // every column has stopped
    if (skip_rec != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *skip_rec = 1;
    return;
  }
  __shared__ cx<R> As[kGemmBK][BM];
  __shared__ cx<R> Bs[kGemmBK][BN];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t row0 = (int64_t)blockIdx.y * BM;
  const int col0 = blockIdx.x * BN;
  cx<R> acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = mk<R>(0, 0);

  for (int64_t k0 = 0; k0 < n; k0 += kGemmBK) {
#pragma unroll
    for (int e = 0; e < A_PER; ++e) {
      const int idx = threadIdx.x + e * kBlock;
      const int ar = idx / kGemmBK, ak = idx % kGemmBK;   // A: row-major reads along k
      const int64_t gr = row0 + ar, gk = k0 + ak;
      As[ak][ar] = (gr < n && gk < n) ? A[gr * lda + gk] : mk<R>(0, 0);
    }
#pragma unroll
    for (int e = 0; e < B_PER; ++e) {
      const int idx = threadIdx.x + e * kBlock;
      const int bk = idx / BN, bc = idx % BN;             // B: rows of k values
      const int64_t gbk = k0 + bk;
      const int gc = col0 + bc;
      Bs[bk][bc] = (gbk < n && gc < k) ? B[gbk * k + gc] : mk<R>(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGemmBK; ++kk) {
      cx<R> a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gr = row0 + ty * TM + i;
    if (gr >= n) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gc = col0 + tx * TN + j;
      if (gc < k) C[gr * k + gc] = acc[i][j];
    }
  }
}

// Column-major user block (column c at U[c * ld .. c * ld + n)) <-> row-major
// internal block (row i at V[i * k .. i * k + k)), with precision change.
template <class Rin, class Rout>
__global__ void block_to_rows(const cx<Rin>* __restrict__ U, int64_t ld, cx<Rout>* __restrict__ V, int64_t n, int k) {
  __shared__ cx<Rin> tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 8 rows of 32 threads
  for (int r = ty; r < 32; r += 8) {
    const int c = c0 + r;
    const int64_t i = i0 + tx;
    if (c < k && i < n) tile[r][tx] = U[(int64_t)c * ld + i];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r;
    const int c = c0 + tx;
    if (c < k && i < n) {
      const cx<Rin> v = tile[tx][r];
      V[i * k + c] = mk<Rout>((Rout)v.x, (Rout)v.y);
    }
  }
}
template <class Rin, class Rout>
__global__ void rows_to_block(const cx<Rin>* __restrict__ V, cx<Rout>* __restrict__ U, int64_t ld, int64_t n, int k) {
  __shared__ cx<Rin> tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r;
    const int c = c0 + tx;
    if (c < k && i < n) tile[r][tx] = V[i * k + c];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int c = c0 + r;
    const int64_t i = i0 + tx;
    if (c < k && i < n) {
      const cx<Rin> v = tile[tx][r];
      U[(int64_t)c * ld + i] = mk<Rout>((Rout)v.x, (Rout)v.y);
    }
  }
}

}  // namespace ccg
