// Exact-integer block products on the bf16 tensor cores (an Ozaki-style
// scheme of digit slices): Y = A X for a block of k right-hand sides, as
// accurate as a GEMM in the operands' own precision -- FP64 for complex128
// (8 digits), FP32 for complex64 (4 digits).  Used for the complex128
// residuals of the batched refinement, its exact complex64 residuals,
// batched solves and ccg_block_matvec.
//
// With the complex product read as one real GEMM (Ah = A as a real n x 2n
// matrix, Xh the 2n x 2k matrix with columns (re x_c, -im x_c) and
// (im x_c, re x_c), as for the split-bf16 product), every row i of Ah is
// scaled by 2^-e_i and every column pair c of Xh by 2^-f_c so that its
// entries lie in (-1, 1), and each scaled entry is cut into S signed
// digits:
//     a = sum_t d_t 2^(-7(t+1)) + rho,   |rho| <= 2^(-7S-1),
// the balanced base-128 digits of the integer N = rint(2^(7S) a), taken of
// |N| and signed: |d_t| <= 64 for t >= 1, |d_0| <= 128, all exactly
// representable in bf16.  Then
//     (Ah Xh)_ic = 2^(e_i + f_c) sum_l 2^(-7(l + 2)) L_l,
//     L_l = sum over digit pairs t + u = l of D^A_t D^X_u   (integer GEMMs),
// truncated at l = S - 1 (S (S + 1) / 2 pairs: 36 for S = 8, whose dropped
// levels are below 2^-54 of 2^(e_i + f_c) per term; 10 for S = 4, below
// 2^-26).  The tensor cores form each level's integer sum in an fp32
// accumulator, exactly: a pair product is at most 2^14 (2^13 with one
// leading digit, 2^12 with none), so a level's products are at most
// 2.5 * 2^14 (1.5 * 2^14 for S = 4), and over a chunk of K = 256 (K = 512)
// its sum stays below 2^23.4 (2^23.6); fp32 represents every integer up to
// 2^24.  After each chunk the epilogue warps read the levels and fold them,
// as exact integers, into int64 accumulators per output,
//     A = sum_{l<4} L_l 2^(7(3-l)),   B = sum_{l>=4} L_l 2^(7(7-l))
// (below 2^52 for K <= 2^16), and at the end
//     (Ah Xh)_ic = 2^(e_i + f_c - 35) A + 2^(e_i + f_c - 63) B
// with one rounding (a second one to float for complex64).  The only other
// errors are the dropped levels and digit remainders.
//
// Kernel: one CTA per 128 x BN output tile (BN = 32 for S = 8, 64 for
// S = 4), 6 warps.  Lane 0 of warp 0 feeds a ring of stages (S digit tiles
// of A, 128 x 32 bf16, and S of X, BN x 32; 64-byte swizzle) with
// cp.async.bulk.tensor; lane 0 of warp 1 issues S tcgen05.mma per K = 16
// step -- A digit t against the X digits 0 .. S - 1 - t stacked along N
// (N = (S - t) BN), into the level accumulators from level t on -- in one
// of two tensor-memory buffers (S levels x BN columns each, 512 columns in
// all), commits each stage and each chunk, so each A digit tile is read
// from shared memory once per step; warps 2-5 read a finished chunk's
// buffer while the next chunk accumulates into the other.  Every mbarrier
// wait is bounded (tcgen05.cuh) and tensor memory is always freed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace ccg {
namespace oz {

constexpr int BM = 128, BK = 32;
constexpr int A_TILE = BM * BK * 2;                 // one A digit tile, bytes
constexpr int THREADS = 192;
constexpr uint32_t TMEM_COLS = 512;                 // 2 buffers x S levels x BN columns
constexpr int64_t kMaxK = 65536;                    // the int64 sums stay below 2^52
constexpr int kNonFinite = 1 << 20;                 // exponent recorded for a row or column with inf / NaN

// S digits per entry (levels t + u = 0 .. S - 1), BN real output columns
// per tile, pipeline stages and K blocks per exact chunk.
template <int S> struct Cfg;
template <> struct Cfg<8> {
  static constexpr int BN = 32, STAGES = 2, CHUNK_KB = 8;    // chunk K = 256; stage 80 KB
};
template <> struct Cfg<4> {
  static constexpr int BN = 64, STAGES = 4, CHUNK_KB = 16;   // chunk K = 512; stage 48 KB
};
template <int S> struct Geo {
  static constexpr int BN = Cfg<S>::BN, STAGES = Cfg<S>::STAGES, CHUNK_KB = Cfg<S>::CHUNK_KB;
  static constexpr int B_TILE = BN * BK * 2;                 // one X digit tile, bytes
  static constexpr int STAGE_BYTES = S * (A_TILE + B_TILE);
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
  static_assert(2 * S * BN == (int)TMEM_COLS, "two buffers of S levels fill tensor memory");
  static_assert(S * BN <= 256, "the stacked X digits fit one MMA's N");
};

template <int S> struct Maps {
  CUtensorMap a[S];
  CUtensorMap x[S];
};

template <int S, class Out>
__global__ void __launch_bounds__(THREADS, 1)
    ozaki_gemm(const __grid_constant__ Maps<S> maps, const int* __restrict__ erow, const int* __restrict__ fcol,
               Out* __restrict__ C, int M, int N, int K, int64_t ldc, int* err, const int* skip, int* skip_rec,
                    long long wait_limit, int withhold) {
  using namespace tc;
  using G = Geo<S>;
  constexpr int LEVELS = S, BN = G::BN, STAGES = G::STAGES, CHUNK_KB = G::CHUNK_KB;
  constexpr int B_TILE = G::B_TILE, STAGE_BYTES = G::STAGE_BYTES;
  if (skip != nullptr && *skip) {  // every column has stopped
    if (skip_rec != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *skip_rec = 1;
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;   // a chunk's levels are in tensor-memory buffer b
  uint64_t* tempty = tfull + 2;       // the epilogue has read buffer b
  uint64_t* done = tempty + 2;        // every MMA has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* verr = err;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int nkb = (K + BK - 1) / BK;
  const int nchunks = (nkb + CHUNK_KB - 1) / CHUNK_KB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;
  if (warp == 0 && lane == 0) {
    // producer: stage s of block kb waits until the MMAs of block kb - STAGES released it
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (kb == withhold) break;  // test hook: this stage's copies are never issued
      if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) & 1) ^ 1, verr, wait_limit)) break;
      unsigned char* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
#pragma unroll
      for (int t = 0; t < S; ++t) {
        tma_load_2d(st + t * A_TILE, &maps.a[t], &full[s], kb * BK, m0);
        tma_load_2d(st + S * A_TILE + t * B_TILE, &maps.x[t], &full[s], kb * BK, n0);
      }
      issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: level l of chunk c accumulates into buffer (c & 1),
    // columns BN l.  One MMA per A digit t covers all its pairs: B is the X
    // digits 0 .. S - 1 - t stacked along N (their tiles are consecutive in
    // the stage, rows BN u .. BN u + BN - 1 for digit u), and D starts at
    // level t, so the product with digit u lands in level t + u.
    for (int kb = 0; kb < nkb; ++kb) {
      const int c = kb / CHUNK_KB, kin = kb - c * CHUNK_KB, b = c & 1;
      if (kin == 0 && c >= 2 && !mbar_wait(&tempty[b], ((c >> 1) - 1) & 1, verr, wait_limit)) break;
      const int s = kb % STAGES;
      if (!mbar_wait(&full[s], (kb / STAGES) & 1, verr, wait_limit)) break;
      fence_after();
      const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint32_t off = kk * 32;  // 16 bf16 along K
        const uint64_t bd = sdesc_k64(base + S * A_TILE + off);
#pragma unroll
        for (int t = 0; t < S; ++t) {
          // t = 0 writes every level first (N = S BN): it alone overwrites
          const uint64_t a = sdesc_k64(base + t * A_TILE + off);
          umma(tmem + (uint32_t)(b * LEVELS * BN + t * BN), a, bd, idesc_bf16(BM, (LEVELS - t) * BN),
               (kin | kk | t) != 0 ? 1u : 0u);
        }
      }
      umma_commit(&empty[s]);
      if (kin == CHUNK_KB - 1 || kb == nkb - 1) umma_commit(&tfull[b]);
    }
    umma_commit(done);  // always: it also tracks every MMA issued before a failure
  } else if (warp >= 2) {
    // epilogue: warp w reads tensor-memory lanes (rows) 32 (w % 4) .. + 31
    const int q = warp & 3;
    const int row = m0 + q * 32 + lane;
    constexpr int NB = S > 4 ? BN : 1;  // the second accumulator only with levels 4 ..
    long long accA[BN], accB[NB];
#pragma unroll
    for (int j = 0; j < BN; ++j) accA[j] = 0;
#pragma unroll
    for (int j = 0; j < NB; ++j) accB[j] = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int b = c & 1;
      ok = __all_sync(0xffffffffu, mbar_wait(&tfull[b], (c >> 1) & 1, verr, wait_limit));
      if (!ok) break;
      fence_after();
#pragma unroll 1
      for (int l = 0; l < LEVELS; ++l) {
        const int sh = 7 * (3 - (l & 3));
#pragma unroll
        for (int h = 0; h < BN / 32; ++h) {
          uint32_t r[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * LEVELS * BN + l * BN + 32 * h), r);
          if (l == LEVELS - 1 && h == BN / 32 - 1) {  // the buffer is free once its last level is in registers
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const long long v = (long long)__float2int_rn(__uint_as_float(r[j])) << sh;
            if (S <= 4 || l < 4) accA[32 * h + j] += v;
            else accB[(32 * h + j) % NB] += v;
          }
        }
      }
    }
    if (ok && __shfl_sync(0xffffffffu, *verr, 0) == 0 && row < M) {
      const int er = erow[row];
      Out* dst = C + (int64_t)row * ldc;
#pragma unroll
      for (int j = 0; j < BN; ++j) {
        const int gc = n0 + j;
        if (gc < N) {
          const int fc = fcol[gc >> 1];
          const int sc = er + fc;
          double v = ldexp((double)accA[j], sc - 35);
          if (S > 4) v += ldexp((double)accB[j % NB], sc - 63);
          if (er >= kNonFinite || fc >= kNonFinite) v = __longlong_as_double(0x7ff8000000000000LL);
          dst[gc] = (Out)v;
        }
      }
    }
  }
  __syncwarp();
  // teardown: no MMA or copy of this CTA may be in flight when it frees its memory
  if (threadIdx.x == 32) mbar_drain(done, 0, verr, wait_limit);
  if (warp == 0 && lane == 0) {
    for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
      mbar_drain(&full[kb % STAGES], (kb / STAGES) & 1, verr, wait_limit);
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// max(m, |v|), with a NaN turned into +inf so that it is not lost.
__device__ __forceinline__ double amax(double m, double v) { return v == v ? fmax(m, fabs(v)) : INFINITY; }

// Exponent ex with m < 2^ex (0 for m = 0; kNonFinite for inf / NaN).
__device__ __forceinline__ int exp_above(double m) {
  if (!(m <= 1.7976931348623157e308)) return kNonFinite;
  int ex = 0;
  if (m > 0.0) frexp(m, &ex);
  return ex;
}

// S signed digits of v 2^(7 - ex) (|v| < 2^ex): N = rint(v 2^(7S - ex)),
// |N| <= 2^(7S); |N| is cut into balanced base-128 digits from the bottom
// (each remainder in [-64, 63], the top digit in [0, 128]) and the sign is
// applied to every digit, so that
//     v = 2^ex sum_t d_t 2^(-7(t+1))
// up to the rounding of N, with |d_t| <= 64 (t >= 1), |d_0| <= 128, and the
// digits of -v the negated digits of v.  Two FP64 operations per value; the
// rest is integer arithmetic.
template <int S>
__device__ __forceinline__ void digits(double v, int ex, __nv_bfloat16 (&d)[S]) {
  const long long Ns = llrint(ldexp(v, 7 * S - ex));
  const int sg = Ns < 0 ? -1 : 1;
  long long N = Ns < 0 ? -Ns : Ns;
#pragma unroll
  for (int t = S - 1; t >= 1; --t) {
    const int r = (int)((N + 64) & 127) - 64;
    d[t] = __int2bfloat16_rn(sg * r);
    N = (N - r) >> 7;
  }
  d[0] = __int2bfloat16_rn(sg * (int)N);
}

// Row exponents (|Ah[i][j]| < 2^e[i]) and the digit slices of the matrix
// read as a real n x 2n matrix; slice t at out + t * n * 2n.  One block per
// row.
template <int S, class R>
__global__ void __launch_bounds__(kBlock) oz_slice_rows(const cx<R>* __restrict__ A, int64_t lda, int64_t n,
                                                        __nv_bfloat16* __restrict__ out, int* __restrict__ e) {
  __shared__ double red[kWarps];
  const int64_t i = blockIdx.x;
  const cx<R>* a = A + i * lda;
  double m = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kBlock) m = amax(amax(m, a[j].x), a[j].y);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) m = fmax(m, red[w]);
  const int ex = exp_above(m);
  if (threadIdx.x == 0) e[i] = ex;
  const int ex_s = ex >= kNonFinite ? 0 : ex;
  const int64_t cnt = n * 2 * n;
  for (int64_t j = threadIdx.x; j < 2 * n; j += kBlock) {
    const cx<R> z = a[j >> 1];
    __nv_bfloat16 d[S];
    digits<S>((double)((j & 1) ? z.y : z.x), ex_s, d);
#pragma unroll
    for (int t = 0; t < S; ++t) out[t * cnt + i * 2 * n + j] = d[t];
  }
}

// Column exponents of the block X (row-major n x k): |re|, |im| of column
// c below 2^f[c].  One block per column.
template <class R>
__global__ void __launch_bounds__(kBlock) oz_col_exp(const cx<R>* __restrict__ X, int64_t n, int k,
                                                     int* __restrict__ f) {
  __shared__ double red[kWarps];
  const int c = blockIdx.x;
  double m = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += kBlock) {
    const cx<R> z = X[j * k + c];
    m = amax(amax(m, (double)z.x), (double)z.y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < kWarps; ++w) mm = fmax(mm, red[w]);
    f[c] = exp_above(mm);
  }
}

// Digit slices of Xh^T (2k rows x 2n): row 2c = (re x_c[j], -im x_c[j])_j,
// row 2c + 1 = (im x_c[j], re x_c[j])_j, each scaled by 2^(7 - f[c]); slice
// t at out + t * 2k * 2n.  32 x 32 tiles through shared memory.
template <int S, class R>
__global__ void oz_slice_block(const cx<R>* __restrict__ X, int64_t n, int k, const int* __restrict__ f,
                               __nv_bfloat16* __restrict__ out) {
  __shared__ cx<R> tile[32][33];
  const int64_t j0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  const int64_t cnt = (int64_t)2 * k * 2 * n;
  for (int r = ty; r < 32; r += 8) {
    const int64_t j = j0 + r;
    const int c = c0 + tx;
    tile[r][tx] = (j < n && c < k) ? X[j * k + c] : cx<R>{R(0), R(0)};
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int c = c0 + r;
    const int64_t j = j0 + tx;
    if (c < k && j < n) {
      const cx<R> z = tile[tx][r];
      const int fx = f[c] >= kNonFinite ? 0 : f[c];
      __nv_bfloat16 dre[S], dim[S];
      digits<S>((double)z.x, fx, dre);
      digits<S>((double)z.y, fx, dim);
      const int64_t e0 = (int64_t)(2 * c) * (2 * n) + 2 * j;  // row 2c
      const int64_t e1 = e0 + 2 * n;                          // row 2c + 1
#pragma unroll
      for (int t = 0; t < S; ++t) {
        __nv_bfloat16* o = out + t * cnt;
        o[e0] = dre[t];
        o[e0 + 1] = __hneg(dim[t]);
        o[e1] = dim[t];
        o[e1 + 1] = dre[t];
      }
    }
  }
}

}  // namespace oz

bool oz_available(const ccg_operator* op) {
  return op->kind == CCG_OPK_DENSE && op->n % 4 == 0 && 2 * op->n <= oz::kMaxK && tc::encoder() != nullptr;
}

// Y = A X (row-major n x k blocks) by the integer-slice scheme on the tensor
// cores, S = 8 digits for complex128 and 4 for complex64.  The matrix digits
// are made on first use and kept with the operator; the block's digits go to
// the handle's staging buffer.
template <class R>
static int oz_product_t(ccg_handle* h, ccg_operator* op, const cx<R>* X, cx<R>* Y, int k, const int* skip) {
  using namespace oz;
  constexpr int S = sizeof(R) == 8 ? 8 : 4;
  using G = Geo<S>;
  const int64_t n = op->n;
  cudaStream_t s = h->stream;
  const size_t abytes = (size_t)n * 2 * n * sizeof(__nv_bfloat16);
  if (!op->oz_ready) {
    op->oz_stream = s;  // stream-ordered: freeing never synchronises the device
    if (cudaMallocAsync(&op->oz_a, S * abytes + 256 + (size_t)n * sizeof(int), s) != cudaSuccess) {
      cudaGetLastError();
      op->oz_a = nullptr;
      set_error("exact tensor-core operand allocation failed");
      return CCG_ERR_NOMEM;
    }
    __nv_bfloat16* slices = static_cast<__nv_bfloat16*>(op->oz_a);
    int* e = reinterpret_cast<int*>(static_cast<char*>(op->oz_a) + S * abytes + 256);
    oz_slice_rows<S, R><<<(unsigned)n, kBlock, 0, s>>>(static_cast<const cx<R>*>(op->A), op->lda, n, slices, e);
    ++h->launches;
    for (int t = 0; t < S; ++t)
      if (!tc::make_map(reinterpret_cast<CUtensorMap*>(op->oz_map[t]), reinterpret_cast<char*>(slices) + t * abytes, n,
                        2 * n, BM, BK)) {
        set_error("cuTensorMapEncodeTiled failed for the matrix digits");
        return CCG_ERR_CUDA;
      }
    op->oz_ready = true;
  }
  const int* erow = reinterpret_cast<const int*>(static_cast<char*>(op->oz_a) + S * abytes + 256);
  // staging: error flag (256 B), column exponents, then S digit slices of Xh^T
  const size_t fbytes = ((size_t)k * sizeof(int) + 255) / 256 * 256;
  const size_t xb = (size_t)2 * k * 2 * n * sizeof(__nv_bfloat16);
  const size_t need = 256 + fbytes + S * xb;
  if (h->oz_bytes < need) {
    if (h->oz_buf) {
      cudaStreamSynchronize(s);
      cudaFree(h->oz_buf);
      h->oz_buf = nullptr;
      h->oz_bytes = 0;
    }
    if (cudaMalloc(&h->oz_buf, need) != cudaSuccess) {
      cudaGetLastError();
      h->oz_buf = nullptr;
      set_error("exact tensor-core staging allocation failed");
      return CCG_ERR_NOMEM;
    }
    h->oz_bytes = need;
    cudaMemsetAsync(h->oz_buf, 0, 256, s);
  }
  int* err = static_cast<int*>(h->oz_buf);
  int* fcol = reinterpret_cast<int*>(static_cast<char*>(h->oz_buf) + 256);
  __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(static_cast<char*>(h->oz_buf) + 256 + fbytes);
  oz_col_exp<R><<<k, kBlock, 0, s>>>(X, n, k, fcol);
  dim3 sg((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32));
  oz_slice_block<S, R><<<sg, kBlock, 0, s>>>(X, n, k, fcol, xs);
  Maps<S> maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int t = 0; t < S; ++t) {
    std::memcpy(&maps.a[t], op->oz_map[t], sizeof(CUtensorMap));
    if (!tc::make_map(&maps.x[t], reinterpret_cast<char*>(xs) + t * xb, 2 * k, 2 * n, G::BN, BK)) {
      set_error("cuTensorMapEncodeTiled failed for the block digits");
      return CCG_ERR_CUDA;
    }
  }
  // once per process: a function-local static is initialised exactly once,
  // also when several threads (serving slots) make their first product together
  static const cudaError_t attr =
      cudaFuncSetAttribute(ozaki_gemm<S, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
  if (attr != cudaSuccess) {
    set_error("exact tensor-core kernel: shared memory opt-in failed");
    return CCG_ERR_CUDA;
  }
  const int Nr = 2 * k;
  dim3 grid((unsigned)((Nr + G::BN - 1) / G::BN), (unsigned)((n + BM - 1) / BM));
  ozaki_gemm<S, R><<<grid, THREADS, G::SMEM_BYTES, s>>>(maps, erow, fcol, reinterpret_cast<R*>(Y), (int)n, Nr,
                                                        (int)(2 * n), (int64_t)Nr, err, skip, timing_rec(h),
                                                        h->wait_limit, h->test_withhold == 1 ? 0 : -1);
  h->launches += 3;
  return cudaGetLastError() == cudaSuccess ? CCG_OK : CCG_ERR_CUDA;
}

int oz_block_product(ccg_handle* h, const ccg_operator* op, const double2* X, double2* Y, int k, const int* skip) {
  return oz_product_t<double>(h, const_cast<ccg_operator*>(op), X, Y, k, skip);
}
int oz_block_product(ccg_handle* h, const ccg_operator* op, const float2* X, float2* Y, int k, const int* skip) {
  return oz_product_t<float>(h, const_cast<ccg_operator*>(op), X, Y, k, skip);
}

// Error flag of the exact tensor-core pipeline: read and clear.
int oz_check_error(ccg_handle* h) {
  if (!h->oz_buf) return CCG_OK;
  int e = 0;
  if (cudaMemcpy(&e, h->oz_buf, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CCG_ERR_CUDA;
  if (e) {
    cudaMemsetAsync(h->oz_buf, 0, sizeof(int), h->stream);
    set_error("exact tensor-core pipeline wait timed out");
    return CCG_ERR_TIMEOUT;
  }
  return CCG_OK;
}

void oz_free(ccg_operator* op) {
  if (op->oz_a) cudaFreeAsync(op->oz_a, op->oz_stream);
  op->oz_a = nullptr;
  op->oz_ready = false;
}

}  // namespace ccg
