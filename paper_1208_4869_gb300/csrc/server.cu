// Serving engine: solve requests of mixed sizes admitted to worker slots as
// slots and device memory (an HBM budget) free up.  Each slot is a host
// thread with its own handle and CUDA stream, so the work of admitted
// requests overlaps on the GPU; a request keeps its Krylov state on its slot
// until it finishes.  Admission is first come, first served: the head of the
// queue waits until its estimated bytes fit the budget (or nothing else is
// running), so a large request is never starved by small ones behind it.
//
// Requests carry a seed instead of data: the dense matrix and right-hand
// sides are generated on the device with Philox4x32-10 (Salmon, Moraes, Dror,
// Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) and Box-Muller;
// dipole requests reuse operators cached per slot and lattice edge.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "workspace.cuh"

namespace ccg {

// ---------------------------------------------------------------------------
// Philox4x32-10: 4 x 32-bit counter, 2 x 32-bit key, ten rounds of
// (hi, lo) = M * x products mixed with the key, key bumped by the Weyl
// constants between rounds.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint64_t p0 = (uint64_t)M0 * c.x, p1 = (uint64_t)M1 * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    U4 o;
    o.x = hi1 ^ c.y ^ k0;
    o.y = lo1;
    o.z = hi0 ^ c.w ^ k1;
    o.w = lo0;
    c = o;
  }
  return c;
}

// Complex normal number (re, im ~ N(0, 1/2)) for element `index` of stream
// `stream` under `seed`: Box-Muller on two uniforms in (0, 1).
__device__ __forceinline__ double2 complex_normal(uint64_t seed, uint32_t stream, uint64_t index) {
  U4 c = {(uint32_t)index, (uint32_t)(index >> 32), stream, 0u};
  const U4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = ((double)(((uint64_t)r.x << 21) ^ (r.y >> 11)) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = ((double)(((uint64_t)r.z << 21) ^ (r.w >> 11)) + 0.5) * (1.0 / 9007199254740992.0);
  const double rad = sqrt(-log(u1));   // sqrt(-2 ln u1) / sqrt(2)
  double s, co;
  sincospi(2.0 * u2, &s, &co);
  return make_double2(rad * co, rad * s);
}

// A = (shift + 0.5 + 0.5i) I + G / sqrt(n), row-major, in both precisions.
__global__ void gen_dense(double2* __restrict__ A64, float2* __restrict__ A32, int64_t n, double shift, uint64_t seed) {
  const double scale = 1.0 / sqrt((double)n);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    double2 a = complex_normal(seed, 0u, (uint64_t)e);
    a.x *= scale;
    a.y *= scale;
    if (e / n == e % n) { a.x += shift + 0.5; a.y += 0.5; }
    A64[e] = a;
    A32[e] = make_float2((float)a.x, (float)a.y);
  }
}
// k complex-normal right-hand sides, column-major n x k.
__global__ void gen_rhs(double2* __restrict__ Y, int64_t n, int k, uint64_t seed) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x)
    Y[e] = complex_normal(seed, 1u, (uint64_t)e);
}
__global__ void to_c64(const double2* __restrict__ a, float2* __restrict__ b, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = make_float2((float)a[e].x, (float)a[e].y);
}
__global__ void to_c128(const float2* __restrict__ a, double2* __restrict__ b, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = make_double2((double)a[e].x, (double)a[e].y);
}

}  // namespace ccg

using namespace ccg;

namespace {

using Clock = std::chrono::steady_clock;

struct Entry {
  ccg_request req;
  ccg_result res;
  bool done = false;
  std::vector<double2> x;
};

struct DipoleOps {
  ccg_operator* op64 = nullptr;
  ccg_operator* op32 = nullptr;
  std::vector<double2> y;  // plane wave
};

}  // namespace

struct ccg_server {
  int device = 0;
  uint64_t budget = 0, used = 0;
  // dense requests of order <= batch_n (0: none) are solved together, up to
  // batch_max right-hand sides per launch (ccg_solve_multi_refined)
  int64_t batch_n = 2048;
  int batch_max = 256;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int64_t> queue;
  std::map<int64_t, std::shared_ptr<Entry>> entries;
  int64_t next_ticket = 1;
  bool stop = false;
  int running = 0;
  int ready = 0;  // slots whose stream and handle exist
  std::vector<std::thread> workers;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Device bytes of the complex128 and complex64 dipole operators of an L^3
// lattice that a slot caches: per precision three FFT grids of (2L)^3
// points and the field-tensor octant of 6 (L+1)^3 components, plus the
// site-index grids and twiddle tables.
// Loosest tolerance that still needs complex128 residuals: a complex64
// solve's own residual carries single-precision rounding of ~1e-6 relative on
// the dipole operators, so it certifies only tolerances of 1e-5 and above.
constexpr double kSingleTol = 1e-5;

uint64_t dipole_op_bytes(int L) {
  const double G = 8.0 * L * L * L, O = 6.0 * (L + 1.0) * (L + 1.0) * (L + 1.0);
  return (uint64_t)((3.0 * G + O) * (16 + 8) + 2.0 * 4.0 * L * L * L + 6.0 * 2 * L * 16);
}

// Device bytes a request holds while it runs (matrices, blocks, workspace);
// for a dipole request also its operators, which the slot that runs it
// keeps cached afterwards (charged to the budget for as long as it does).
uint64_t estimate_bytes(const ccg_request& r) {
  if (r.kind == CCG_REQ_DIPOLE) {
    const double N3 = 3.0 * 0.55 * r.L * r.L * r.L;
    return (uint64_t)(40.0 * N3 * 16) + dipole_op_bytes(r.L);
  }
  const double n = (double)r.n, k = std::max(1, r.nrhs);
  // complex128 and complex64 matrices, the split-bf16 terms, the fixed-point
  // digits of the complex128 matrix, blocks and workspace
  double b = 16 * n * n + 8 * n * n + 8 * n * n + 16 * n * n + 40.0 * n * std::max(k, 8.0) * 16 + 64.0 * n * 16;
  // batched requests also keep the exact products' digit slices of both
  // matrices (8 and 4 bf16 slices of n x 2n) where those products apply
  if (k > 1 && r.n % 4 == 0 && 2 * r.n <= 65536) b += 32 * n * n + 16 * n * n;
  return (uint64_t)b;
}

int run_dense(ccg_handle* h, cudaStream_t s, const ccg_request& r, ccg_result& res, std::vector<double2>* xout) {
  const int64_t n = r.n;
  const int k = std::max(1, r.nrhs);
  double2 *A64 = nullptr, *Y = nullptr, *X = nullptr;
  float2 *A32 = nullptr, *Y32 = nullptr, *X32 = nullptr;
  const bool single = r.tol >= kSingleTol && r.mode == 0;
  auto freeall = [&]() {
    for (void* p : {(void*)A64, (void*)A32, (void*)Y, (void*)X, (void*)Y32, (void*)X32})
      if (p) cudaFreeAsync(p, s);
  };
  if (cudaMallocAsync(&A64, (size_t)n * n * sizeof(double2), s) != cudaSuccess ||
      cudaMallocAsync(&A32, (size_t)n * n * sizeof(float2), s) != cudaSuccess ||
      cudaMallocAsync(&Y, (size_t)n * k * sizeof(double2), s) != cudaSuccess ||
      cudaMallocAsync(&X, (size_t)n * k * sizeof(double2), s) != cudaSuccess ||
      (single && (cudaMallocAsync(&Y32, (size_t)n * k * sizeof(float2), s) != cudaSuccess ||
                  cudaMallocAsync(&X32, (size_t)n * k * sizeof(float2), s) != cudaSuccess))) {
    cudaGetLastError();
    freeall();
    set_error("server: request allocation failed");
    return CCG_ERR_NOMEM;
  }
  gen_dense<<<2048, kBlock, 0, s>>>(A64, A32, n, r.shift, r.seed);
  gen_rhs<<<512, kBlock, 0, s>>>(Y, n, k, r.seed);
  cudaMemsetAsync(X, 0, (size_t)n * k * sizeof(double2), s);
  ccg_operator *op64 = nullptr, *op32 = nullptr;
  int st = ccg_op_dense(h, CCG_C128, n, A64, n, 0, &op64);
  if (st == CCG_OK) st = ccg_op_dense(h, CCG_C64, n, A32, n, 0, &op32);
  const int maxit = r.maxit > 0 ? r.maxit : 1000;
  if (st == CCG_OK && r.mode == 1) {
    // baseline: complex128 solves, one right-hand side at a time
    res.iters = 0;
    res.relres = 0.0;
    for (int c = 0; c < k && st >= 0; ++c) {
      ccg_info info;
      const int sc = ccg_solve(h, CCG_BICGSTAB, op64, Y + (int64_t)c * n, X + (int64_t)c * n, r.tol, maxit, nullptr,
                               &info);
      st = std::max(st, sc);
      if (sc < 0) st = sc;
      res.iters = std::max(res.iters, info.iters);
      res.relres = std::max(res.relres, info.true_relres);
    }
  } else if (st == CCG_OK) {
    if (single) {
      to_c64<<<512, kBlock, 0, s>>>(Y, Y32, n * k);
      cudaMemsetAsync(X32, 0, (size_t)n * k * sizeof(float2), s);
      if (k == 1) {
        ccg_info info;
        st = ccg_solve(h, CCG_BICGSTAB, op32, Y32, X32, r.tol, maxit, nullptr, &info);
        res.iters = info.iters;
        res.relres = info.true_relres;
      } else {
        std::vector<int32_t> it(k);
        std::vector<double> rr(k);
        st = ccg_solve_batched(h, CCG_BICGSTAB, op32, k, Y32, n, X32, n, r.tol, maxit, it.data(), nullptr, rr.data());
        res.iters = *std::max_element(it.begin(), it.end());
        res.relres = *std::max_element(rr.begin(), rr.end());
      }
      to_c128<<<512, kBlock, 0, s>>>(X32, X, n * k);
    } else if (k == 1) {
      ccg_info info;
      int inner = 0;
      st = ccg_solve_refined(h, CCG_BICGSTAB, op64, op32, Y, X, r.tol, 30, 1e-5, maxit, nullptr, &inner, &info);
      res.iters = info.iters;
      res.relres = info.true_relres;
    } else {
      std::vector<int32_t> outer(k);
      std::vector<double> rr(k);
      st = ccg_solve_batched_refined(h, CCG_BICGSTAB, op64, op32, k, Y, n, X, n, r.tol, 30, 1e-5, maxit, outer.data(),
                                     nullptr, nullptr, rr.data());
      res.iters = *std::max_element(outer.begin(), outer.end());
      res.relres = *std::max_element(rr.begin(), rr.end());
    }
  }
  if (xout) {
    xout->resize((size_t)n * k);
    cudaMemcpyAsync(xout->data(), X, (size_t)n * k * sizeof(double2), cudaMemcpyDeviceToHost, s);
  }
  cudaStreamSynchronize(s);
  if (op64) ccg_op_destroy(op64);
  if (op32) ccg_op_destroy(op32);
  freeall();
  cudaStreamSynchronize(s);
  res.n = n;
  res.nrhs = k;
  return st;
}

// Small dense requests solved together: every right-hand side of every
// request is one system of a ccg_solve_multi_refined launch (the requests'
// matrices and blocks generated as in run_dense); results per request are
// the worst status and the largest iteration count and residual of its
// columns.  Returns the launch's status (per-request statuses in res).
int run_dense_batch(ccg_handle* h, cudaStream_t s, std::vector<std::shared_ptr<Entry>>& batch) {
  const size_t m = batch.size();
  std::vector<double2*> A64(m, nullptr), Y(m, nullptr), X(m, nullptr);
  std::vector<float2*> A32(m, nullptr);
  std::vector<ccg_operator*> o64(m, nullptr), o32(m, nullptr);
  std::vector<const ccg_operator*> ops, ops_in;
  std::vector<const void*> yv;
  std::vector<void*> xv;
  std::vector<double> tol;
  std::vector<size_t> owner;
  int st = CCG_OK;
  int maxit = 1000;
  for (size_t q = 0; q < m && st == CCG_OK; ++q) {
    const ccg_request& r = batch[q]->req;
    const int64_t n = r.n;
    const int k = std::max(1, r.nrhs);
    if (r.maxit > 0) maxit = std::min(maxit, r.maxit);
    if (cudaMallocAsync(&A64[q], (size_t)n * n * sizeof(double2), s) != cudaSuccess ||
        cudaMallocAsync(&A32[q], (size_t)n * n * sizeof(float2), s) != cudaSuccess ||
        cudaMallocAsync(&Y[q], (size_t)n * k * sizeof(double2), s) != cudaSuccess ||
        cudaMallocAsync(&X[q], (size_t)n * k * sizeof(double2), s) != cudaSuccess) {
      cudaGetLastError();
      set_error("server: request allocation failed");
      st = CCG_ERR_NOMEM;
      break;
    }
    gen_dense<<<2048, kBlock, 0, s>>>(A64[q], A32[q], n, r.shift, r.seed);
    gen_rhs<<<512, kBlock, 0, s>>>(Y[q], n, k, r.seed);
    cudaMemsetAsync(X[q], 0, (size_t)n * k * sizeof(double2), s);
    st = ccg_op_dense(h, CCG_C128, n, A64[q], n, 0, &o64[q]);
    if (st == CCG_OK) st = ccg_op_dense(h, CCG_C64, n, A32[q], n, 0, &o32[q]);
    for (int c = 0; c < k && st == CCG_OK; ++c) {
      ops.push_back(o64[q]);
      ops_in.push_back(o32[q]);
      yv.push_back(Y[q] + (int64_t)c * n);
      xv.push_back(X[q] + (int64_t)c * n);
      tol.push_back(r.tol);
      owner.push_back(q);
    }
  }
  const size_t cnt = ops.size();
  std::vector<int32_t> outer(cnt, 0), sts(cnt, 0);
  std::vector<double> rr(cnt, 0.0);
  if (st == CCG_OK)
    st = ccg_solve_multi_refined(h, CCG_BICGSTAB, (int64_t)cnt, ops.data(), ops_in.data(), yv.data(), xv.data(),
                                 tol.data(), 30, 1e-5, maxit, outer.data(), nullptr, sts.data(), rr.data());
  for (size_t q = 0; q < m; ++q) {
    ccg_result& res = batch[q]->res;
    res.status = st < 0 ? st : CCG_OK;
    res.iters = 0;
    res.relres = 0.0;
    res.n = batch[q]->req.n;
    res.nrhs = std::max(1, batch[q]->req.nrhs);
  }
  if (st >= 0) {
    for (size_t c = 0; c < cnt; ++c) {
      ccg_result& res = batch[owner[c]]->res;
      res.iters = std::max(res.iters, outer[c]);
      res.relres = std::max(res.relres, rr[c]);
      if (sts[c] < 0) res.status = std::min(res.status, sts[c]);
      else if (res.status >= 0) res.status = std::max(res.status, sts[c]);
    }
  }
  for (size_t q = 0; q < m; ++q) {
    if (batch[q]->req.keep_x && X[q] && st >= 0) {
      batch[q]->x.resize((size_t)batch[q]->req.n * std::max(1, batch[q]->req.nrhs));
      cudaMemcpyAsync(batch[q]->x.data(), X[q], batch[q]->x.size() * sizeof(double2), cudaMemcpyDeviceToHost, s);
    }
  }
  cudaStreamSynchronize(s);
  for (size_t q = 0; q < m; ++q) {
    if (o64[q]) ccg_op_destroy(o64[q]);
    if (o32[q]) ccg_op_destroy(o32[q]);
    for (void* p : {(void*)A64[q], (void*)A32[q], (void*)Y[q], (void*)X[q]})
      if (p) cudaFreeAsync(p, s);
  }
  cudaStreamSynchronize(s);
  return st;
}

int run_dipole(ccg_handle* h, cudaStream_t s, std::map<int, DipoleOps>& cache, const ccg_request& r, ccg_result& res,
               std::vector<double2>* xout, bool* created) {
  const int L = r.L;
  auto it = cache.find(L);
  *created = false;
  if (it == cache.end()) {
    DipoleOps d;
    std::vector<uint8_t> occ((size_t)L * L * L);
    const double c = (L - 1) / 2.0, R2 = (L / 2.0) * (L / 2.0);
    std::vector<int> zs;
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j)
        for (int l = 0; l < L; ++l) {
          const double d2 = (i - c) * (i - c) + (j - c) * (j - c) + (l - c) * (l - c);
          const bool in = d2 <= R2;
          occ[((size_t)i * L + j) * L + l] = in ? 1 : 0;
          if (in) zs.push_back(l);
        }
    int st = ccg_op_dipole(h, CCG_C128, L, L, L, occ.data(), r.kd, r.m_re, r.m_im, &d.op64);
    if (st == CCG_OK) st = ccg_op_dipole(h, CCG_C64, L, L, L, occ.data(), r.kd, r.m_re, r.m_im, &d.op32);
    if (st != CCG_OK) {
      if (d.op64) ccg_op_destroy(d.op64);
      return st;
    }
    const size_t N = zs.size();
    d.y.assign(3 * N, make_double2(0.0, 0.0));
    for (size_t q = 0; q < N; ++q) {
      const std::complex<double> e = std::polar(1.0, r.kd * zs[q]);
      d.y[q] = make_double2(e.real(), e.imag());
    }
    it = cache.emplace(L, std::move(d)).first;
    *created = true;
  }
  DipoleOps& d = it->second;
  const int64_t n = (int64_t)d.y.size();
  double2 *Y = nullptr, *X = nullptr;
  float2 *Y32 = nullptr, *X32 = nullptr;
  const bool single = r.tol >= kSingleTol && r.mode == 0;
  cudaMallocAsync(&Y, n * sizeof(double2), s);
  cudaMallocAsync(&X, n * sizeof(double2), s);
  if (single) {
    cudaMallocAsync(&Y32, n * sizeof(float2), s);
    cudaMallocAsync(&X32, n * sizeof(float2), s);
  }
  if (cudaGetLastError() != cudaSuccess) {
    set_error("server: request allocation failed");
    return CCG_ERR_NOMEM;
  }
  cudaMemcpyAsync(Y, d.y.data(), n * sizeof(double2), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(X, 0, n * sizeof(double2), s);
  const int maxit = r.maxit > 0 ? r.maxit : 3000;
  ccg_info info;
  int st;
  if (r.mode == 1) {
    st = ccg_solve(h, CCG_COCG, d.op64, Y, X, r.tol, maxit, nullptr, &info);
    res.iters = info.iters;
  } else if (single) {
    to_c64<<<512, kBlock, 0, s>>>(Y, Y32, n);
    cudaMemsetAsync(X32, 0, n * sizeof(float2), s);
    st = ccg_solve(h, CCG_COCG, d.op32, Y32, X32, r.tol, maxit, nullptr, &info);
    to_c128<<<512, kBlock, 0, s>>>(X32, X, n);
    res.iters = info.iters;
  } else {
    int inner = 0;
    st = ccg_solve_refined(h, CCG_COCG, d.op64, d.op32, Y, X, r.tol, 30, 1e-4, maxit, nullptr, &inner, &info);
    res.iters = info.iters;
  }
  res.relres = info.true_relres;
  if (xout) {
    xout->resize(n);
    cudaMemcpyAsync(xout->data(), X, n * sizeof(double2), cudaMemcpyDeviceToHost, s);
  }
  for (void* p : {(void*)Y, (void*)X, (void*)Y32, (void*)X32})
    if (p) cudaFreeAsync(p, s);
  cudaStreamSynchronize(s);
  res.n = n;
  res.nrhs = 1;
  return st;
}

void worker(ccg_server* sv, int slot) {
  cudaSetDevice(sv->device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  ccg_handle* h = nullptr;
  ccg_create(&h, s);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    ++sv->ready;
  }
  sv->cv.notify_all();
  std::map<int, DipoleOps> cache;
  uint64_t cached_bytes = 0;   // budget charged for this slot's cached operators
  // systems one many-system launch of this slot's handle takes
  const int capacity = h ? std::min(pk_capacity(h, CCG_BICGSTAB, CCG_C64), pk_capacity(h, M_REFRES, CCG_C128)) : 0;
  // only single-right-hand-side requests: a request's right-hand sides become
  // systems of their own in the many-system launch, each sweeping the matrix
  // again, while the per-slot block solver reads it once for all of them
  // (measured: 3x slower to batch the stream's 1-64 right-hand-side requests)
  auto batchable = [&](const ccg_request& r) {
    return r.kind == CCG_REQ_DENSE && r.mode == 0 && r.n <= sv->batch_n && r.nrhs <= 1 && capacity >= 1;
  };
  for (;;) {
    std::shared_ptr<Entry> e;
    std::vector<std::shared_ptr<Entry>> batch;
    uint64_t bytes = 0;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv.wait(lk, [&] {
        if (sv->queue.empty()) return sv->stop;
        const uint64_t b = estimate_bytes(sv->entries[sv->queue.front()]->req);
        return sv->used + b <= sv->budget || sv->running == 0;
      });
      if (sv->queue.empty()) break;
      const int64_t t = sv->queue.front();
      sv->queue.pop_front();
      e = sv->entries[t];
      bytes = estimate_bytes(e->req);
      sv->used += bytes;
      ++sv->running;
      e->res.t_start = sv->now();
      e->res.slot = slot;
      if (batchable(e->req)) {
        // take every other queued small dense request that fits the launch
        // and the budget, in queue order
        batch.push_back(e);
        int systems = std::max(1, e->req.nrhs);
        const int cap = std::min(capacity, sv->batch_max);
        for (auto it = sv->queue.begin(); it != sv->queue.end();) {
          const std::shared_ptr<Entry>& o = sv->entries[*it];
          const uint64_t ob = estimate_bytes(o->req);
          const int k = std::max(1, o->req.nrhs);
          if (batchable(o->req) && systems + k <= cap && sv->used + ob <= sv->budget) {
            systems += k;
            sv->used += ob;
            bytes += ob;
            o->res.t_start = e->res.t_start;
            o->res.slot = slot;
            batch.push_back(o);
            it = sv->queue.erase(it);
          } else {
            ++it;
          }
        }
      }
    }
    sv->cv.notify_all();
    if (!batch.empty()) {
      const int st = h ? run_dense_batch(h, s, batch) : CCG_ERR_CUDA;
      std::lock_guard<std::mutex> lk(sv->mu);
      const double t = sv->now();
      for (auto& b : batch) {
        if (st < 0) b->res.status = st;
        b->res.t_done = t;
        b->done = true;
      }
      sv->used -= bytes;
      --sv->running;
      sv->cv.notify_all();
      continue;
    }
    std::vector<double2>* xo = e->req.keep_x ? &e->x : nullptr;
    int st = h ? CCG_OK : CCG_ERR_CUDA;
    bool created = false;
    if (st == CCG_OK)
      st = e->req.kind == CCG_REQ_DIPOLE ? run_dipole(h, s, cache, e->req, e->res, xo, &created)
                                         : run_dense(h, s, e->req, e->res, xo);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      e->res.status = st;
      e->res.t_done = sv->now();
      e->done = true;
      sv->used -= bytes;
      // operators this slot now caches stay charged until the slot exits
      if (created) {
        const uint64_t ob = dipole_op_bytes(e->req.L);
        sv->used += ob;
        cached_bytes += ob;
      }
      --sv->running;
    }
    sv->cv.notify_all();
  }
  for (auto& kv : cache) {
    ccg_op_destroy(kv.second.op64);
    ccg_op_destroy(kv.second.op32);
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->used -= cached_bytes;
  }
  if (h) ccg_destroy(h);
  cudaStreamDestroy(s);
}

}  // namespace

extern "C" {

ccg_status ccg_server_create(ccg_server** out, int device, int slots, uint64_t budget) {
  if (!out || slots < 1 || slots > 32) { set_error("ccg_server_create: need 1 <= slots <= 32"); return CCG_ERR_INVALID; }
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    set_error("ccg_server_create: no such CUDA device");
    return CCG_ERR_CUDA;
  }
  // keep memory freed by finished requests in the device's pool for the next ones
  cudaMemPool_t pool;
  if (cudaSetDevice(device) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  ccg_server* sv = new ccg_server();
  sv->device = device;
  sv->budget = budget ? budget : (uint64_t)120 << 30;
  sv->t0 = Clock::now();
  for (int i = 0; i < slots; ++i) sv->workers.emplace_back(worker, sv, i);
  {
    // return once every slot can take work, so that slot set-up is not
    // charged to the first requests' latency
    std::unique_lock<std::mutex> lk(sv->mu);
    sv->cv.wait(lk, [&] { return sv->ready == slots; });
  }
  *out = sv;
  return CCG_OK;
}

ccg_status ccg_server_submit(ccg_server* sv, const ccg_request* r, int64_t* ticket) {
  if (!sv || !r || !ticket) { set_error("ccg_server_submit: NULL argument"); return CCG_ERR_INVALID; }
  if (r->kind == CCG_REQ_DENSE && (r->n < 1 || r->nrhs < 1 || r->nrhs > 256 || r->n % 4 != 0)) {
    set_error("ccg_server_submit: dense requests need n >= 4 (a multiple of 4) and 1 <= nrhs <= 256");
    return CCG_ERR_INVALID;
  }
  if (r->kind == CCG_REQ_DIPOLE && (r->L < 1 || r->L > 128)) {
    set_error("ccg_server_submit: dipole requests need 1 <= L <= 128");
    return CCG_ERR_INVALID;
  }
  if (r->kind != CCG_REQ_DENSE && r->kind != CCG_REQ_DIPOLE) { set_error("ccg_server_submit: bad kind"); return CCG_ERR_INVALID; }
  if (!(r->tol > 0.0)) { set_error("ccg_server_submit: need tol > 0"); return CCG_ERR_INVALID; }
  auto e = std::make_shared<Entry>();
  e->req = *r;
  std::memset(&e->res, 0, sizeof(e->res));
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    e->res.t_submit = sv->now();
    *ticket = sv->next_ticket++;
    sv->entries[*ticket] = e;
    sv->queue.push_back(*ticket);
  }
  sv->cv.notify_all();
  return CCG_OK;
}

ccg_status ccg_server_poll(ccg_server* sv, int64_t ticket, int* done) {
  if (!sv || !done) return CCG_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->entries.find(ticket);
  if (it == sv->entries.end()) { set_error("ccg_server_poll: unknown ticket"); return CCG_ERR_INVALID; }
  *done = it->second->done ? 1 : 0;
  return CCG_OK;
}

ccg_status ccg_server_wait(ccg_server* sv, int64_t ticket, ccg_result* res, void* x) {
  if (!sv) return CCG_ERR_INVALID;
  std::shared_ptr<Entry> e;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->entries.find(ticket);
    if (it == sv->entries.end()) { set_error("ccg_server_wait: unknown ticket"); return CCG_ERR_INVALID; }
    e = it->second;
    sv->cv.wait(lk, [&] { return e->done; });
    sv->entries.erase(it);
  }
  if (res) *res = e->res;
  if (x && !e->x.empty()) std::memcpy(x, e->x.data(), e->x.size() * sizeof(double2));
  return CCG_OK;
}

double ccg_server_now(const ccg_server* sv) { return sv ? sv->now() : 0.0; }

ccg_status ccg_server_set_batching(ccg_server* sv, int64_t max_n, int max_systems) {
  if (!sv || max_n < 0 || max_systems < 1) {
    set_error("ccg_server_set_batching: need a server, max_n >= 0 and max_systems >= 1");
    return CCG_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->batch_n = max_n;
  sv->batch_max = max_systems;
  return CCG_OK;
}

ccg_status ccg_server_estimate(const ccg_request* r, uint64_t* bytes) {
  if (!r || !bytes) { set_error("ccg_server_estimate: NULL argument"); return CCG_ERR_INVALID; }
  if (r->kind != CCG_REQ_DENSE && r->kind != CCG_REQ_DIPOLE) { set_error("ccg_server_estimate: bad kind"); return CCG_ERR_INVALID; }
  *bytes = estimate_bytes(*r);
  return CCG_OK;
}

ccg_status ccg_server_charged(ccg_server* sv, uint64_t* bytes) {
  if (!sv || !bytes) { set_error("ccg_server_charged: NULL argument"); return CCG_ERR_INVALID; }
  std::lock_guard<std::mutex> lk(sv->mu);
  *bytes = sv->used;
  return CCG_OK;
}

ccg_status ccg_server_destroy(ccg_server* sv) {
  if (!sv) return CCG_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (auto& t : sv->workers) t.join();
  delete sv;
  return CCG_OK;
}

}  // extern "C"
