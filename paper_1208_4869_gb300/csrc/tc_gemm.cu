// Tensor-core block product for complex64 operators: Y = A X for a block of
// k right-hand sides, on the 5th-generation tensor cores (tcgen05) with
// operands staged by TMA and the accumulator in tensor memory.
//
// The complex product is one real GEMM: with the interleaved complex matrix
// read as a real n x 2n matrix Ah (row i = re a_i0, im a_i0, re a_i1, ...),
// and the real 2n x 2k matrix Xh whose columns 2c and 2c+1 are
// (re x_c, -im x_c) and (im x_c, re x_c) interleaved the same way,
//     Yh = Ah Xh
// is the interleaved complex block Y (row-major n x k).  Single precision
// is carried by operands split into T bf16 terms (a = a_0 + a_1 [+ a_2],
// a_0 = bf16(a), a_t = bf16(a - a_0 - ... - a_{t-1})) and the products of
// order below T accumulated in fp32 in tensor memory:
//   T = 2: A0 X0 + A0 X1 + A1 X0                    (~2^-17 relative)
//   T = 3: A0 X0 + A0 X1 + A1 X0 + A0 X2 + A1 X1 + A2 X0   (~2^-24, fp32 level)
//
// Kernel: output tiles of 128 x BN (BN = 256 for T = 2, 128 for T = 3),
// 6 warps.  Lane 0 of warp 0 feeds a 4-stage ring of shared-memory tiles (T
// tiles of A, 128 x 32 bf16, and T of X, BN x 32; 64-byte swizzle) with
// cp.async.bulk.tensor and mbarrier transaction counts; lane 0 of warp 1
// issues the tcgen05.mma of every product and K = 16 step of a stage,
// releases the stage with tcgen05.commit and alternates between two
// accumulators in tensor memory; warps 2-5 read a finished accumulator with
// tcgen05.ld while the next one fills.
//
// Schedule (stream-K): a row unit is one K block (32) of one row block; the
// R = row blocks x K blocks units, in row-block order, are cut into P equal
// ranges (+-1), P = SMs / column tiles, and range p goes to the ncol CTAs
// p * ncol + c, one per column tile c, which therefore read the same A rows
// at the same time.  Every SM gets the same work whatever the number of
// tiles (at n = 8192, k = 256: 128 tiles, 152 SMs).  A range cuts at most its
// last row block short; that piece is computed first and its fp32 partial
// tile published (per-warp flags carrying the launch's epoch), the pieces
// that end a tile last: the CTA holding a tile's last K block adds the
// partials of the lower ranges, in order of K, to its own.  Waits go only to
// lower-numbered CTAs, which start no later, and are bounded like every
// mbarrier wait: a wait that gives up records an error flag and lets the CTA
// finish (tensor memory is always freed), so a fault in the pipeline cannot
// hang the GPU.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace ccg {
namespace tc {

constexpr int BM = 128, BK = 32, STAGES = 4, THREADS = 192;
constexpr int MIN_UNITS = 32;  // K blocks per range at least (fewer ranges on small products)
template <int T> struct Cfg {
  static constexpr int BN = T == 2 ? 256 : 128;
  static constexpr int A_TILE = BM * BK * 2;         // bytes of one bf16 A tile
  static constexpr int B_TILE = BN * BK * 2;         // bytes of one bf16 X tile
  static constexpr int STAGE_BYTES = T * (A_TILE + B_TILE);
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
  static constexpr uint32_t TMEM_COLS = 2 * BN;      // two accumulators
  static constexpr int NPROD = T == 2 ? 3 : 6;       // products of order below T
};
// (term of A, term of X) of each product
__device__ constexpr int kProdA[6] = {0, 0, 1, 0, 1, 2};
__device__ constexpr int kProdX[6] = {0, 1, 0, 2, 1, 0};

struct TcMaps {
  CUtensorMap a[3];
  CUtensorMap x[3];
};

// The stream-K cut: ranges [begin(p), begin(p + 1)) of the R row units.
struct Split {
  int nrb, nkb, ncol, P;
  __host__ __device__ int64_t begin(int p) const { return (int64_t)nrb * nkb * p / P; }
};

// The cut for an n x n operator, k right-hand sides and `sms` SMs (one CTA
// per SM): P ranges of row units, ncol column tiles each.
template <int T> static Split make_split(int64_t n, int k, int sms) {
  Split sp;
  sp.nrb = (int)((n + BM - 1) / BM);
  sp.nkb = (int)((2 * n + BK - 1) / BK);
  sp.ncol = (2 * k + Cfg<T>::BN - 1) / Cfg<T>::BN;
  const int64_t units = (int64_t)sp.nrb * sp.nkb;
  sp.P = (int)std::min<int64_t>(std::max(1, sms / sp.ncol), std::max<int64_t>(1, units / MIN_UNITS));
  return sp;
}

// Segments of range [u0, u1) (one per row block it touches).
__host__ __device__ __forceinline__ int segments(const Split& sp, int64_t u0, int64_t u1) {
  return (int)((u1 - 1) / sp.nkb - u0 / sp.nkb) + 1;
}

// Segment si of range [u0, u1): its row block and K blocks [kb0, kb1).  The
// last row block (the only one a range can cut short) comes first.
struct Seg {
  int r, kb0, kb1;
};
__host__ __device__ __forceinline__ Seg segment(const Split& sp, int64_t u0, int64_t u1, int si) {
  const int rlo = (int)(u0 / sp.nkb), rhi = (int)((u1 - 1) / sp.nkb);
  const int r = si == 0 ? rhi : rlo + si - 1;
  const int64_t base = (int64_t)r * sp.nkb;
  Seg g;
  g.r = r;
  g.kb0 = (int)((u0 > base ? u0 : base) - base);
  g.kb1 = (int)((u1 < base + sp.nkb ? u1 : base + sp.nkb) - base);
  return g;
}

// The lowest range holding K blocks of row block r, for the range p that
// finishes it: ranges first .. p - 1 hold its earlier K blocks.
__host__ __device__ __forceinline__ int first_contributor(const Split& sp, int p, int r) {
  const int64_t rs = (int64_t)r * sp.nkb;
  int pf = p - 1;
  while (sp.begin(pf) > rs) --pf;
  return pf;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Bounded wait for a flag to carry this launch's epoch (false and the error
// flag set when it runs out or another thread gave up).
__device__ __forceinline__ bool flag_wait(const unsigned* f, unsigned epoch, volatile int* err, long long limit) {
  const long long t0 = clock64();
  while (ld_acquire(f) != epoch) {
    if (*err) return false;
    if (clock64() - t0 > limit) {
      *err = 1;
      return false;
    }
  }
  return true;
}

// C (M x N fp32, leading dimension ldc) = sum of the split products.
// work: one BM x BN fp32 partial tile per CTA (column-major); flags: 4 per
// CTA (one per epilogue warp), holding the epoch of the launch that last
// published that warp's rows.
template <int T>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_bf16_split(const __grid_constant__ TcMaps maps, float* __restrict__ C, int M, int N, int K, int64_t ldc,
                    Split sp, float* __restrict__ work, unsigned* flags, unsigned epoch, int* err,
                    const int* skip, int* skip_rec, long long wait_limit, int withhold, int nopub) {
  using G = Cfg<T>;
  constexpr int BN = G::BN;
  if (skip != nullptr && *skip) {  // every column has stopped
    if (skip_rec != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *skip_rec = 1;
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * G::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;  // accumulator b holds a finished segment
  uint64_t* tempty = tfull + 2;      // the epilogue has read accumulator b
  uint64_t* done = tempty + 2;       // every MMA has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* verr = err;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int cta = blockIdx.x, p = cta / sp.ncol, ct = cta - p * sp.ncol;
  const int n0 = ct * BN;
  const int64_t u0 = sp.begin(p), u1 = sp.begin(p + 1);
  const int nseg = segments(sp, u0, u1);

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
                 "r"(G::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;
  if (warp == 0 && lane == 0) {
    // producer: the g-th K block of this CTA uses stage g % STAGES, which
    // the MMAs of K block g - STAGES released
    int g = 0;
    bool go = true;
    for (int si = 0; si < nseg && go; ++si) {
      const Seg sg = segment(sp, u0, u1, si);
      const int m0 = sg.r * BM;
      for (int kb = sg.kb0; kb < sg.kb1; ++kb, ++g) {
        const int s = g % STAGES;
        // (g == withhold: test hook, no copies from this K block on)
        if (g == withhold || (g >= STAGES && !mbar_wait(&empty[s], ((g / STAGES) & 1) ^ 1, verr, wait_limit))) {
          go = false;
          break;
        }
        unsigned char* st = smem + s * G::STAGE_BYTES;
        mbar_expect_tx(&full[s], G::STAGE_BYTES);
#pragma unroll
        for (int t = 0; t < T; ++t) {
          tma_load_2d(st + t * G::A_TILE, &maps.a[t], &full[s], kb * BK, m0);
          tma_load_2d(st + T * G::A_TILE + t * G::B_TILE, &maps.x[t], &full[s], kb * BK, n0);
        }
        issued = g + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: segment si accumulates into buffer si & 1
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    int g = 0;
    bool ok = true;
    for (int si = 0; si < nseg && ok; ++si) {
      const Seg sg = segment(sp, u0, u1, si);
      const int b = si & 1;
      if (si >= 2 && !mbar_wait(&tempty[b], ((si >> 1) - 1) & 1, verr, wait_limit)) break;
      const uint32_t acc = tmem + (uint32_t)(b * BN);
      for (int kb = sg.kb0; kb < sg.kb1; ++kb, ++g) {
        const int s = g % STAGES;
        if (!mbar_wait(&full[s], (g / STAGES) & 1, verr, wait_limit)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t base = smem_u32(smem + s * G::STAGE_BYTES);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t off = kk * 32;  // 16 bf16 along K
#pragma unroll
          for (int q = 0; q < G::NPROD; ++q) {
            const uint64_t a = sdesc_k64(base + kProdA[q] * G::A_TILE + off);
            const uint64_t bd = sdesc_k64(base + T * G::A_TILE + kProdX[q] * G::B_TILE + off);
            umma(acc, a, bd, idesc, (kb != sg.kb0 || kk != 0 || q != 0) ? 1u : 0u);
          }
        }
        umma_commit(&empty[s]);
      }
      umma_commit(&tfull[b]);  // also after a failure: it tracks the MMAs issued
    }
    umma_commit(done);
  } else if (warp >= 2) {
    // epilogue: warp w reads tensor-memory lanes (rows) 32 (w % 4) .. + 31
    const int q = warp & 3, rt = q * 32 + lane;
    for (int si = 0; si < nseg; ++si) {
      const Seg sg = segment(sp, u0, u1, si);
      const int b = si & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(&tfull[b], (si >> 1) & 1, verr, wait_limit))) break;
      fence_after();
      const bool last = sg.kb1 == sp.nkb;  // this CTA finishes the tile
      // the lower ranges holding K blocks of this tile: pf .. p - 1
      int pf = p;
      if (last && sg.kb0 > 0) {
        pf = first_contributor(sp, p, sg.r);
        bool ok = true;
        for (int pp = pf; pp < p && ok; ++pp) ok = flag_wait(&flags[(pp * sp.ncol + ct) * 4 + q], epoch, verr, wait_limit);
        if (!__all_sync(0xffffffffu, ok)) break;
      }
      if (__shfl_sync(0xffffffffu, *verr, 0) != 0) break;
      const int row = sg.r * BM + rt;
#pragma unroll 1
      for (int h = 0; h < BN / 32; ++h) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + 32 * h), r);
        if (h == BN / 32 - 1) {  // the accumulator is free once its last columns are in registers
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[b]);
        }
        if (!last) {
          float* w = work + (size_t)cta * BM * BN + (size_t)(32 * h) * BM + rt;
#pragma unroll
          for (int j = 0; j < 32; ++j) w[(size_t)j * BM] = __uint_as_float(r[j]);
        } else {
          float v[32];
          if (pf < p) {
            const float* w = work + (size_t)(pf * sp.ncol + ct) * BM * BN + (size_t)(32 * h) * BM + rt;
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = __ldcg(w + (size_t)j * BM);
            for (int pp = pf + 1; pp < p; ++pp) {
              w = work + (size_t)(pp * sp.ncol + ct) * BM * BN + (size_t)(32 * h) * BM + rt;
#pragma unroll
              for (int j = 0; j < 32; ++j) v[j] += __ldcg(w + (size_t)j * BM);
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] += __uint_as_float(r[j]);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
          }
          if (row < M) {
            float* dst = C + (int64_t)row * ldc + n0 + 32 * h;
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (n0 + 32 * h + j < N) dst[j] = v[j];
          }
        }
      }
      if (!last && !(nopub && p == 0)) {  // publish this warp's rows of the partial tile
        // (nopub: test hook, range 0 never publishes, so its finisher's wait runs out)
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(&flags[cta * 4 + q], epoch);
      }
    }
  }
  __syncwarp();
  // teardown: no MMA or copy of this CTA may be in flight when it frees its memory
  if (threadIdx.x == 32) mbar_drain(done, 0, verr, wait_limit);
  if (warp == 0 && lane == 0) {
    for (int g = issued > STAGES ? issued - STAGES : 0; g < issued; ++g)
      mbar_drain(&full[g % STAGES], (g / STAGES) & 1, verr, wait_limit);
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::TMEM_COLS) : "memory");
}

// Split v into T bf16 terms (t[0] = bf16(v), t[i] = bf16(v - t[0] - ... )).
template <int T> __device__ __forceinline__ void split_terms(float v, __nv_bfloat16 (&t)[3]) {
  float rem = v;
#pragma unroll
  for (int i = 0; i < T; ++i) {
    t[i] = __float2bfloat16_rn(rem);
    rem -= __bfloat162float(t[i]);
  }
}

// The interleaved complex64 matrix (row i at A + i * lda complex) as T bf16
// terms of the real n x 2n matrix, term t at out + t * n * 2n.
template <int T>
__global__ void split_matrix(const float2* __restrict__ A, int64_t lda, int64_t n, __nv_bfloat16* __restrict__ out) {
  const int64_t count = n * 2 * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / (2 * n), jj = e - i * 2 * n;
    const float2 a = A[i * lda + (jj >> 1)];
    __nv_bfloat16 t[3];
    split_terms<T>((jj & 1) ? a.y : a.x, t);
#pragma unroll
    for (int q = 0; q < T; ++q) out[q * count + e] = t[q];
  }
}

// Xh^T as T bf16 terms (2k rows x 2n, term t at out + t * 2k * 2n) from the
// row-major block X (n x k complex): row 2c = (re x_c[j], -im x_c[j])_j,
// row 2c + 1 = (im x_c[j], re x_c[j])_j.
template <int T>
__global__ void split_block(const float2* __restrict__ X, int64_t n, int k, __nv_bfloat16* __restrict__ out) {
  __shared__ float2 tile[32][33];
  const int64_t j0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  const int64_t count = (int64_t)2 * k * 2 * n;
  for (int r = ty; r < 32; r += 8) {
    const int64_t j = j0 + r;
    const int c = c0 + tx;
    tile[r][tx] = (j < n && c < k) ? X[j * k + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int c = c0 + r;
    const int64_t j = j0 + tx;
    if (c < k && j < n) {
      const float2 x = tile[tx][r];
      const float vals[4] = {x.x, -x.y, x.y, x.x};  // (2c, 2j), (2c, 2j+1), (2c+1, 2j), (2c+1, 2j+1)
      // each row's pair (2j, 2j + 1) as one 4-byte store (coalesced across the warp)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t e = (int64_t)(2 * c + h) * (2 * n) + 2 * j;
        __nv_bfloat16 t0[3], t1[3];
        split_terms<T>(vals[2 * h], t0);
        split_terms<T>(vals[2 * h + 1], t1);
#pragma unroll
        for (int i = 0; i < T; ++i) {
          __nv_bfloat162 pr;
          pr.x = t0[i];
          pr.y = t1[i];
          *reinterpret_cast<__nv_bfloat162*>(out + i * count + e) = pr;
        }
      }
    }
  }
}

}  // namespace tc

bool tc_available(const ccg_operator* op) {
  return op->kind == CCG_OPK_DENSE && op->dtype == CCG_C64 && op->n % 4 == 0 && tc::encoder() != nullptr;
}

template <int T>
static int tc_product_t(ccg_handle* h, ccg_operator* op, const float2* X, float2* Y, int k, const int* skip) {
  using G = tc::Cfg<T>;
  const int64_t n = op->n;
  cudaStream_t s = h->stream;
  const size_t abytes = (size_t)n * 2 * n * sizeof(__nv_bfloat16);
  if (op->tc_ready && op->tc_terms != T) tc_free(op);
  if (!op->tc_ready) {
    op->tc_stream = s;  // stream-ordered: freeing never synchronises the device
    if (cudaMallocAsync(&op->tc_ahi, T * abytes, s) != cudaSuccess) {
      cudaGetLastError();
      op->tc_ahi = nullptr;
      set_error("tensor-core operand allocation failed");
      return CCG_ERR_NOMEM;
    }
    tc::split_matrix<T><<<2048, kBlock, 0, s>>>(static_cast<const float2*>(op->A), op->lda, n,
                                                 static_cast<__nv_bfloat16*>(op->tc_ahi));
    for (int t = 0; t < T; ++t)
      if (!tc::make_map(reinterpret_cast<CUtensorMap*>(op->tc_map[t]), static_cast<char*>(op->tc_ahi) + t * abytes, n,
                        2 * n, tc::BM, tc::BK)) {
        set_error("cuTensorMapEncodeTiled failed for the matrix");
        return CCG_ERR_CUDA;
      }
    op->tc_terms = T;
    op->tc_ready = true;
  }
  // the handle's staging: error flag (256 B), the ranges' flags (4 per CTA),
  // the T bf16 terms of Xh^T (2k x 2n each), one partial tile per CTA
  const int Nr = 2 * k;
  const tc::Split sp = tc::make_split<T>(n, k, h->num_sms);
  const int ctas = sp.P * sp.ncol;
  const size_t flag_bytes = ((size_t)ctas * 4 * sizeof(unsigned) + 255) / 256 * 256;
  const size_t xb = (size_t)2 * k * 2 * n * sizeof(__nv_bfloat16);
  const size_t xoff = 256 + flag_bytes;
  const size_t woff = (xoff + T * xb + 255) / 256 * 256;
  const size_t need = woff + (size_t)ctas * tc::BM * G::BN * sizeof(float);
  if (h->tc_bytes < need) {
    if (h->tc_buf) {
      cudaStreamSynchronize(s);
      cudaFree(h->tc_buf);
      h->tc_buf = nullptr;
      h->tc_bytes = 0;
    }
    if (cudaMalloc(&h->tc_buf, need) != cudaSuccess) {
      cudaGetLastError();
      h->tc_buf = nullptr;
      set_error("tensor-core staging allocation failed");
      return CCG_ERR_NOMEM;
    }
    h->tc_bytes = need;
    h->tc_flag_bytes = 0;
  }
  char* buf = static_cast<char*>(h->tc_buf);
  if (h->tc_flag_bytes < flag_bytes) {  // flags never written yet hold no epoch (0)
    cudaMemsetAsync(buf, 0, 256 + flag_bytes, s);
    h->tc_flag_bytes = flag_bytes;
  }
  if (++h->tc_epoch == 0) h->tc_epoch = 1;
  int* err = reinterpret_cast<int*>(buf);
  unsigned* flags = reinterpret_cast<unsigned*>(buf + 256);
  __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(buf + xoff);
  float* work = reinterpret_cast<float*>(buf + woff);
  dim3 sg((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32));
  tc::split_block<T><<<sg, kBlock, 0, s>>>(X, n, k, xs);
  tc::TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int t = 0; t < T; ++t) {
    std::memcpy(&maps.a[t], op->tc_map[t], sizeof(CUtensorMap));
    if (!tc::make_map(&maps.x[t], reinterpret_cast<char*>(xs) + t * xb, 2 * k, 2 * n, G::BN, tc::BK)) {
      set_error("cuTensorMapEncodeTiled failed for the block");
      return CCG_ERR_CUDA;
    }
  }
  // once per process: a function-local static is initialised exactly once,
  // also when several threads (serving slots) make their first product together
  static const cudaError_t attr =
      cudaFuncSetAttribute(tc::gemm_bf16_split<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
  if (attr != cudaSuccess) {
    set_error("tensor-core kernel: shared memory opt-in failed");
    return CCG_ERR_CUDA;
  }
  tc::gemm_bf16_split<T><<<ctas, tc::THREADS, G::SMEM_BYTES, s>>>(
      maps, reinterpret_cast<float*>(Y), (int)n, Nr, (int)(2 * n), (int64_t)Nr, sp, work, flags, h->tc_epoch, err,
      skip, timing_rec(h), h->wait_limit, h->test_withhold == 1 ? 0 : -1, h->test_withhold == 2);
  h->launches += 2;
  return cudaGetLastError() == cudaSuccess ? CCG_OK : CCG_ERR_CUDA;
}

// Y = A X (row-major n x k complex64 blocks) on the tensor cores with the
// handle's split (2 or 3 bf16 terms).
int tc_block_product(ccg_handle* h, const ccg_operator* op_c, const float2* X, float2* Y, int k, const int* skip) {
  ccg_operator* op = const_cast<ccg_operator*>(op_c);
  return h->tc_terms == 2 ? tc_product_t<2>(h, op, X, Y, k, skip) : tc_product_t<3>(h, op, X, Y, k, skip);
}

namespace tc {
// Host run of the cut the product uses (launcher and kernel functions), with
// every invariant the kernel relies on checked; returns the violations.
template <int T> static int64_t check_cut(int64_t n, int k, int sms, int* ctas_out) {
  const Split sp = make_split<T>(n, k, sms);
  const int ctas = sp.P * sp.ncol;
  *ctas_out = ctas;
  int64_t bad = 0;
  const int64_t units = (int64_t)sp.nrb * sp.nkb;
  // computed[(tile) * nkb + kb], tile = r * ncol + c; published[tile]: ranges
  // that left a piece of the tile unfinished; finished[tile]: its finishers
  std::vector<unsigned char> computed((size_t)units * sp.ncol, 0);
  std::vector<std::vector<int>> published((size_t)sp.nrb * sp.ncol);
  std::vector<int> finished((size_t)sp.nrb * sp.ncol, 0);
  struct Fin { int p, c, r, pf; };
  std::vector<Fin> fins;
  if (sp.P < 1 || sp.ncol * Cfg<T>::BN < 2 * k) ++bad;
  for (int cta = 0; cta < ctas; ++cta) {
    const int p = cta / sp.ncol, c = cta - p * sp.ncol;
    const int64_t u0 = sp.begin(p), u1 = sp.begin(p + 1);
    if (!(u1 > u0)) { ++bad; continue; }
    const int nseg = segments(sp, u0, u1);
    for (int si = 0; si < nseg; ++si) {
      const Seg g = segment(sp, u0, u1, si);
      if (g.r < 0 || g.r >= sp.nrb || g.kb0 < 0 || g.kb0 >= g.kb1 || g.kb1 > sp.nkb) { ++bad; continue; }
      const size_t tile = (size_t)g.r * sp.ncol + c;
      for (int kb = g.kb0; kb < g.kb1; ++kb) {
        if (computed[tile * sp.nkb + kb]++) ++bad;  // a unit computed twice
        if ((int64_t)kb * BK >= 2 * n) ++bad;       // a K block past the operator
      }
      if (g.kb1 < sp.nkb) {
        if (si != 0) ++bad;  // only a range's first segment may be unfinished
        published[tile].push_back(p);
      } else {
        ++finished[tile];
        const int pf = g.kb0 > 0 ? first_contributor(sp, p, g.r) : p;
        if (pf < 0 || pf > p) ++bad;
        fins.push_back({p, c, g.r, pf});
      }
    }
  }
  for (size_t u = 0; u < computed.size(); ++u)
    if (computed[u] != 1) ++bad;  // a unit missed (or counted above)
  for (size_t t = 0; t < finished.size(); ++t)
    if (finished[t] != 1) ++bad;  // a tile with no or several finishers
  for (const Fin& f : fins) {
    // the finisher waits for ranges pf .. p - 1, lower CTAs whose unfinished
    // pieces of this tile are exactly those
    std::vector<int> want;
    for (int q = f.pf; q < f.p; ++q) want.push_back(q);
    std::vector<int> got = published[(size_t)f.r * sp.ncol + f.c];
    std::sort(got.begin(), got.end());
    if (got != want) ++bad;
    for (int q : want)
      if (q * sp.ncol + f.c >= f.p * sp.ncol + f.c || (q * sp.ncol + f.c) * 4 + 3 >= ctas * 4) ++bad;
  }
  return bad;
}
}  // namespace tc

// Error flag of the tensor-core pipeline (a bounded wait gave up): read and clear.
int tc_check_error(ccg_handle* h) {
  if (!h->tc_buf) return CCG_OK;
  int e = 0;
  if (cudaMemcpy(&e, h->tc_buf, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CCG_ERR_CUDA;
  if (e) {
    cudaMemsetAsync(h->tc_buf, 0, sizeof(int), h->stream);
    set_error("tensor-core pipeline wait timed out");
    return CCG_ERR_TIMEOUT;
  }
  return CCG_OK;
}

void tc_free(ccg_operator* op) {
  if (op->tc_ahi) cudaFreeAsync(op->tc_ahi, op->tc_stream);
  op->tc_ahi = nullptr;
  op->tc_ready = false;
  op->tc_terms = 0;
}

}  // namespace ccg

extern "C" ccg_status ccg_check_block_schedule(int64_t n, int k, int terms, int sms, int* ctas, int64_t* bad) {
  if (n < 1 || k < 1 || k > 256 || (terms != 2 && terms != 3) || sms < 1 || !ctas || !bad) {
    ccg::set_error("ccg_check_block_schedule: need n >= 1, 1 <= k <= 256, terms 2 or 3, sms >= 1, outputs");
    return CCG_ERR_INVALID;
  }
  try {
    *bad = terms == 2 ? ccg::tc::check_cut<2>(n, k, sms, ctas) : ccg::tc::check_cut<3>(n, k, sms, ctas);
  } catch (const std::bad_alloc&) {
    ccg::set_error("ccg_check_block_schedule: host allocation failed");
    return CCG_ERR_NOMEM;
  }
  return CCG_OK;
}
