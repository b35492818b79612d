// Krylov iterations on the GPU: BiCGSTAB, CGNR, QMR, BiCG, GMRES(m), CGS,
// CGNE, TFQMR (Sec. 2.1, the PIM methods), the complex-symmetric CG (Sec.
// 2.2), BiCGstab(l) (Sec. 3.1) and COCR (Sec. 3.4), unpreconditioned.
//
// One iteration is a fixed sequence of kernels on the handle's stream:
// operator sweeps (gemv.cuh) and "phase" kernels.  A phase kernel makes one
// pass over the vectors doing a method's elementwise updates, accumulates
// the dot products the next step needs, reduces them in a single pass over
// the grid (common.cuh), and in the last block computes the method's scalar
// recurrences into the device SolveState.  Scalars never travel to the host
// during a solve.  Every kernel first reads SolveState::poll.done and returns
// at once when the solve has stopped, so the host may enqueue iterations
// ahead of the convergence test and only polls a small record every few
// iterations.
//
// Readings of the methods (the manual prints no recurrences): stopping on
// ||r_k|| / ||y|| <= tol with the recurrence residual; shadow vectors equal
// to r_0; BiCGSTAB's half-step exit on ||s||; QMR with A^H and conjugated
// products; COCG with the unconjugated form [u, v] = sum u_i v_i.  Dot
// products accumulate in double at both precisions, and the scalars are
// formed in double and rounded to the working precision for the vector
// updates.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <functional>
#include <memory>

#include "common.cuh"
#include "reduce.cuh"
#include "gemv.cuh"
#include "internal.h"
#include "phases.cuh"
#include "workspace.cuh"
#include "fx.cuh"

namespace ccg {

// ---------------------------------------------------------------------------
// GMRES(m) (Saad-Schultz; PIM `rgmres`, Sec. 2.1), complex form.  Arnoldi
// step j orthogonalises w = A v_j against v_0 .. v_j by classical
// Gram-Schmidt applied twice: h1 = V^H w in one pass, w -= V h1 with
// h2 = V^H w in a second, w -= V h2 with ||w|| in a third (three passes and
// three grid reductions per step instead of j + 1 dependent ones; in exact
// arithmetic the same basis and Hessenberg column as modified Gram-Schmidt).
// The last block of the third pass applies the earlier Givens rotations to
// the column, forms the new one and the least-squares residual |g_{j+1}|.
// `half` marks a cycle that stopped early (convergence, the iteration cap):
// its remaining products and passes skip, and the cycle end forms x.
// ---------------------------------------------------------------------------


enum { GM_DOT = 0, GM_UPD_DOT = 1, GM_UPD_NORM = 2 };

// Column j of the Hessenberg matrix after orthogonalisation (||w|| = eta):
// rotations, residual, stopping test.  One thread.
__device__ void gm_column(const GmBuf& b, int j, double eta, SolveState* st) {
  const int m = b.m;
  for (int i = 0; i <= j; ++i) b.H[i * m + j] = cadd(b.H[i * m + j], b.h2[i]);
  for (int i = 0; i < j; ++i) {
    const double2 a = b.H[i * m + j], c = b.H[(i + 1) * m + j];
    b.H[i * m + j] = cadd(cscale(b.cs[i], a), cmul(b.sn[i], c));
    b.H[(i + 1) * m + j] = csub(cscale(b.cs[i], c), cmul(cconj(b.sn[i]), a));
  }
  const double2 a = b.H[j * m + j];
  const double aa = cabs(a);
  const double nu = sqrt(aa * aa + eta * eta);
  if (nu == 0.0) {  // singular projected system: x stays at the cycle start
    set_breakdown(st, CCG_BD_HESS);
    return;
  }
  if (aa == 0.0) {
    b.cs[j] = 0.0;
    b.sn[j] = mkc(1.0, 0.0);
    b.H[j * m + j] = mkc(eta, 0.0);
  } else {
    const double2 ph = cscale(1.0 / aa, a);
    b.cs[j] = aa / nu;
    b.sn[j] = cscale(eta / nu, ph);
    b.H[j * m + j] = cscale(nu, ph);
  }
  b.H[(j + 1) * m + j] = mkc(0.0, 0.0);
  const double2 gj = b.g[j];
  b.g[j + 1] = cscale(-1.0, cmul(cconj(b.sn[j]), gj));
  b.g[j] = cscale(b.cs[j], gj);
  const int k = st->poll.k + 1;
  const double rel = cabs(b.g[j + 1]) / st->poll.ynorm;
  st->poll.k = k;
  st->poll.relres = rel;
  st->hist[k] = rel;
  st->gm_cols = j + 1;
  st->gm_eta = eta;
  bool stop = true;
  if (nonfinite(rel)) st->poll.status = ST_NONFINITE;
  else if (rel <= st->tol) st->poll.status = ST_OK;
  else if (k >= st->maxit) st->poll.status = ST_NOT_CONVERGED;
  else stop = false;
  if (stop) {
    st->half = 1;
    st->gm_final = 1;
  }
}

// One orthogonalisation pass over w and the basis v_0 .. v_j (columns of V,
// leading dimension ldv), E rows per thread kept in registers:
//   GM_DOT       h1 = V^H w into Hessenberg column j;
//   GM_UPD_DOT   w -= V h1, then h2 = V^H w;
//   GM_UPD_NORM  w -= V h2, then ||w|| and the column's rotations.
// The j + 1 dot products reduce per warp by shuffles, per block through
// shared memory, and over the grid in the last block to arrive, in block
// order (deterministic).
template <class R, int E, int MODE>
__global__ void __launch_bounds__(kBlock) gm_pass(const cx<R>* __restrict__ V, int64_t ldv, cx<R>* __restrict__ w,
                                                  int64_t n, int j, GmBuf b, SolveState* st) {
  if (st->poll.done || st->half) return;
  __shared__ double2 red[kMaxBasis + 1][kWarps];
  __shared__ bool is_last;
  const int J = j + 1, m = b.m;
  const int64_t i0 = (int64_t)blockIdx.x * (kBlock * E) + threadIdx.x;
  cx<R> u[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int64_t i = i0 + (int64_t)e * kBlock;
    u[e] = i < n ? w[i] : mk<R>(0, 0);
  }
  if (MODE != GM_DOT) {
    for (int l = 0; l < J; ++l) {
      const cx<R> c = narrow<R>(MODE == GM_UPD_DOT ? b.H[l * m + j] : b.h2[l]);
      const cx<R>* Vl = V + (int64_t)l * ldv;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t i = i0 + (int64_t)e * kBlock;
        if (i < n) u[e] = csub(u[e], cmul(c, Vl[i]));
      }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int64_t i = i0 + (int64_t)e * kBlock;
      if (i < n) w[i] = u[e];
    }
  }
  if (MODE == GM_UPD_NORM) {
    acc_t<R> acc[1];
    acc_zero(acc[0]);
#pragma unroll
    for (int e = 0; e < E; ++e) acc_nrm2(acc, u[e]);
    double tot[1];
    if (grid_reduce<1>(acc, reinterpret_cast<double*>(b.part), b.counter, tot) && threadIdx.x == 0)
      gm_column(b, j, sqrt(tot[0]), st);
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int l = 0; l < J; ++l) {
    const cx<R>* Vl = V + (int64_t)l * ldv;
    acc_t<R> a2[2];
    acc_zero(a2[0]);
    acc_zero(a2[1]);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int64_t i = i0 + (int64_t)e * kBlock;
      if (i < n) acc_dotc(a2, Vl[i], u[e]);
    }
    const double s0 = warp_acc_sum(a2[0]), s1 = warp_acc_sum(a2[1]);
    if (lane == 0) red[l][warp] = mkc(s0, s1);
  }
  __syncthreads();
  const int64_t ld = m + 1;
  for (int t = threadIdx.x; t < J; t += kBlock) {
    double2 sum = mkc(0.0, 0.0);
#pragma unroll
    for (int q = 0; q < kWarps; ++q) sum = cadd(sum, red[t][q]);
    b.part[(int64_t)blockIdx.x * ld + t] = sum;
  }
  __threadfence();
  // Grid sum in a fan-in-kRedGroup tree: at each level the last block of a
  // group sums its group's rows (all loads in flight) into the group's
  // first row; the block that sums the last group holds the total in row 0.
  // Fixed order: deterministic.
  int idx = blockIdx.x, cnt = gridDim.x, stride = 1, base = 0;
  while (cnt > 1) {
    const int g = idx / kRedGroup, g0 = g * kRedGroup;
    const int gsize = min(kRedGroup, cnt - g0);
    __syncthreads();
    if (threadIdx.x == 0) {
      is_last = atomicAdd(&b.counter[base + g], 1u) == (unsigned)gsize - 1u;
      if (is_last) b.counter[base + g] = 0u;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int t = threadIdx.x; t < J; t += kBlock) {
      double2 v[kRedGroup];
#pragma unroll
      for (int q = 0; q < kRedGroup; ++q)
        v[q] = q < gsize ? __ldcg(&b.part[(int64_t)(g0 + q) * stride * ld + t]) : mkc(0.0, 0.0);
      double2 sum = mkc(0.0, 0.0);
#pragma unroll
      for (int q = 0; q < kRedGroup; ++q) sum = cadd(sum, v[q]);
      b.part[(int64_t)g0 * stride * ld + t] = sum;
    }
    __threadfence();
    base += (cnt + kRedGroup - 1) / kRedGroup;
    idx = g;
    cnt = (cnt + kRedGroup - 1) / kRedGroup;
    stride *= kRedGroup;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < J; t += kBlock) {
    const double2 sum = __ldcg(&b.part[t]);
    if (MODE == GM_DOT) b.H[t * m + j] = sum;
    else b.h2[t] = sum;
  }
}

template <class R> struct GmBegin : PhaseBase {  // v_0 = r / beta, g = (beta, 0, ...): a new cycle
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* r;
  cx<R>* v0;
  GmBuf b;
  R binv;
  __device__ __forceinline__ void load(const SolveState* st) { binv = (R)(1.0 / st->gm_beta); }
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) { v0[i] = cscale(binv, r[i]); }
  __device__ void finish(const double*, SolveState* st) {
    b.g[0] = mkc(st->gm_beta, 0.0);
    for (int i = 1; i <= b.m; ++i) b.g[i] = mkc(0.0, 0.0);
    st->gm_cols = 0;
    st->half = 0;
  }
};
template <class R> struct GmScale : PhaseBase {  // v_{j+1} = w / ||w||
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* w;
  cx<R>* v;
  R einv;
  __device__ __forceinline__ bool skip(const SolveState* st) const { return st->half != 0; }
  __device__ __forceinline__ void load(const SolveState* st) { einv = (R)(1.0 / st->gm_eta); }
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) { v[i] = cscale(einv, w[i]); }
  __device__ void finish(const double*, SolveState*) {}
};
// Cycle end: R y = g by back substitution (one thread).  Enqueued after
// every step: at the last step of a cycle (always = 1) it runs while the
// solve is live, elsewhere only once the cycle has stopped early.
__global__ void gm_solve(GmBuf b, SolveState* st, int always) {
  if (st->poll.done || threadIdx.x != 0 || (!always && !st->half)) return;
  const int cols = st->gm_cols, m = b.m;
  for (int i = cols - 1; i >= 0; --i) {
    double2 t = b.g[i];
    for (int l = i + 1; l < cols; ++l) t = csub(t, cmul(b.H[i * m + l], b.yv[l]));
    b.yv[i] = cdiv(t, b.H[i * m + i]);
  }
}
template <class R> struct GmXUpd : PhaseBase {  // x += V y; the solve ends here after a final cycle
  static constexpr int NQ = 1;
  int64_t n;
  cx<R>* x;
  const cx<R>* V;
  int64_t ldv;
  const double2* yv;
  int cols;
  bool always;  // as for gm_solve
  __device__ __forceinline__ bool skip(const SolveState* st) const { return !always && !st->half; }
  __device__ __forceinline__ void load(const SolveState* st) { cols = st->gm_cols; }
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) {
    cx<R> xi = x[i];
    for (int l = 0; l < cols; ++l) xi = cadd(xi, cmul(narrow<R>(yv[l]), V[(int64_t)l * ldv + i]));
    x[i] = xi;
  }
  __device__ void finish(const double*, SolveState* st) {
    if (st->gm_final) st->poll.done = 1;
  }
};
template <class R> struct GmRestart : PhaseBase {  // r = y - A x, beta = ||r||; stop if it meets tol
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* y;
  MvOut<R> ax;
  cx<R>* r;
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> ri = csub(y[i], ax.get(i));
    r[i] = ri;
    acc_nrm2(acc, ri);
  }
  __device__ void finish(const double* t, SolveState* st) {
    const double beta = sqrt(t[0]);
    if (beta / st->poll.ynorm <= st->tol) {
      st->poll.status = ST_OK;
      st->poll.done = 1;
      return;
    }
    st->gm_beta = beta;
  }
};

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
#define CCG_CUDA(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                   \
      return CCG_ERR_CUDA;                                                             \
    }                                                                                  \
  } while (0)

template <class R> struct Runner {
  ccg_handle* h;
  const ccg_operator* op;
  cudaStream_t s;
  Dense<R> d;
  Ws<R> w;
  Red red;
  int grid_vec;
  static constexpr int kDt = sizeof(R) == 8 ? CCG_C128 : CCG_C64;

  Runner(ccg_handle* h_, const ccg_operator* op_, const Ws<R>& w_)
      : h(h_), op(op_), s(h_->stream), d(op_, h_->num_sms), w(w_) {
    red.partials = w.partials;
    red.counter = w.counter;
    grid_vec = phase_grid(h, d.n);
  }

  // A kernel of the loop: with programmatic dependent launch where the handle
  // allows it, so that it starts launching while the previous one finishes
  // (each kernel waits for its predecessor inside, pdl_wait).
  template <class... KArgs, class... Args>
  void launch(void (*kern)(KArgs...), dim3 grid, dim3 block, Args... args) {
    launch_smem(kern, grid, block, 0, args...);
  }
  template <class... KArgs, class... Args>
  void launch_smem(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, Args... args) {
    if (h->pdl) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = grid;
      cfg.blockDim = block;
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, kern, args...);
    } else {
      kern<<<grid, block, smem, s>>>(args...);
    }
    ++h->launches;
  }

  template <class P> void phase(const P& p) { launch(phase_kernel<P, acc_t<R>>, dim3(grid_vec), dim3(kBlock), p, w.st, red); }

  MvOut<R> plain(const cx<R>* y) const { MvOut<R> m; m.y = y; m.P = nullptr; m.ld = d.n; m.nparts = 1; return m; }

  // The operator's fixed-point digits (complex128 dense, integer-pipe sweeps
  // on; made on first use), or null: the FP64 pipe.
  const int4* fx_digits() {
    if (sizeof(R) != 8 || !h->fx_mode || w.xfx == nullptr || !fx_prepare(h, op)) return nullptr;
    return static_cast<const int4*>(op->fx_a);
  }
  const int* fx_rowexp() const {
    return reinterpret_cast<const int*>(static_cast<const char*>(op->fx_a) + (size_t)d.n * d.n * sizeof(int4) + 256);
  }

  // One GMRES orthogonalisation pass of step j over the basis.
  template <int MODE> void gm_pass_launch(cx<R>* wv, int j) {
    const int grid = gm_grid(d.n);
    switch (gm_rows_per_thread(d.n)) {
      case 1: gm_pass<R, 1, MODE><<<grid, kBlock, 0, s>>>(w.basis, w.ldv, wv, d.n, j, w.gm, w.st); break;
      case 2: gm_pass<R, 2, MODE><<<grid, kBlock, 0, s>>>(w.basis, w.ldv, wv, d.n, j, w.gm, w.st); break;
      case 4: gm_pass<R, 4, MODE><<<grid, kBlock, 0, s>>>(w.basis, w.ldv, wv, d.n, j, w.gm, w.st); break;
      default: gm_pass<R, 8, MODE><<<grid, kBlock, 0, s>>>(w.basis, w.ldv, wv, d.n, j, w.gm, w.st); break;
    }
    ++h->launches;
  }

  // y = A x.  timed = false for products the device may skip (x0 = 0), which
  // would otherwise enter the sweep timing with a near-zero duration.
  // A user operator's matvec or cmatvec, enqueued by the caller's function
  // on this stream; the first nonzero return is kept on the handle.
  void callback(bool conj, const cx<R>* x, cx<R>* y) {
    const ccg_matvec_fn f = conj ? op->cb_cmatvec : op->cb_matvec;
    const int rc = f ? f(op->cb_ctx, op->n, x, y, s) : -1;
    if (rc != 0 && h->cb_status == 0) h->cb_status = rc;
  }

  MvOut<R> apply_n(const cx<R>* x, cx<R>* y, const SolveState* st, bool timed = true) {
    if (timed) timing_begin(h);
    int* rec = timed ? timing_rec(h) : nullptr;
    if (op->kind == CCG_OPK_CALLBACK) {
      callback(false, x, y);
    } else if (op->kind == CCG_OPK_DIPOLE) {
      dipole_apply(op, x, y, false, st, s, rec, h->pdl != 0);
      h->launches += op->dip.kernels;
    } else {
      const cx<R>* A = d.A;
      const int64_t lda = d.lda, n = d.n;
      const SolveState* cst = st;
      if constexpr (sizeof(R) == 4) {
        if (d.unit == 2) launch(gemv_n_rows<R, 2, kRowSplit>, dim3(d.grid_rows), dim3(kBlock), A, lda, n, x, y, cst, rec);
        else launch(gemv_n_rows<R, 1, kRowSplit>, dim3(d.grid_rows), dim3(kBlock), A, lda, n, x, y, cst, rec);
      } else if (const int4* C = fx_digits()) {
        // the integer-pipe sweep: the vector's digits, then the rows from the
        // operator's digit copy (both launches inside the sweep's timing)
        const int* rowexp = fx_rowexp();
        const int4* xd = w.xfx;
        const int* meta = w.xmeta;
        launch(fx_split_vector<1024, false>, dim3(1), dim3(1024), x, n, w.xfx, w.xmeta, cst, rowexp);
        launch(gemv_fx_rows<kFxSplit>, dim3(d.grid_fx), dim3(kBlock), A, lda, C, rowexp, n, x, xd, meta, y, cst, rec);
      } else {
        launch(gemv_n_rows<R, 1, kRowSplit>, dim3(d.grid_rows), dim3(kBlock), A, lda, n, x, y, cst, rec);
      }
    }
    if (timed) timing_end(h, kDt, CCG_SWEEP_N, d.sweep_bytes());
    return plain(y);
  }
  // A^H x: dense operators leave nsplit partial vectors in P2; others write y.
  MvOut<R> apply_c(const cx<R>* x, cx<R>* y, const SolveState* st) {
    timing_begin(h);
    int* rec = timing_rec(h);
    if (op->kind == CCG_OPK_CALLBACK) {
      callback(true, x, y);
      timing_end(h, kDt, CCG_SWEEP_C, d.sweep_bytes());
      return plain(y);
    }
    if (op->kind == CCG_OPK_DIPOLE) {
      dipole_apply(op, x, y, true, st, s, rec, h->pdl != 0);
      h->launches += op->dip.kernels;
      timing_end(h, kDt, CCG_SWEEP_C, d.sweep_bytes());
      return plain(y);
    }
    dim3 grid(d.ncb, d.tc.nsplit);
    const int64_t rpr = d.tc.rows_per_range;
    const cx<R>* A = d.A;
    const int64_t lda = d.lda, n = d.n;
    const SolveState* cst = st;
    cx<R>* P2 = w.P2;
    if constexpr (sizeof(R) == 4) {
      if (d.unit == 2) launch(gemv_tile_h<R, 2, Dense<R>::E>, grid, dim3(kBlock), A, lda, n, rpr, x, P2, cst, rec);
      else launch(gemv_tile_h<R, 1, Dense<R>::E>, grid, dim3(kBlock), A, lda, n, rpr, x, P2, cst, rec);
    } else if (const int4* C = fx_digits()) {
      // the integer-pipe sweep: the row-scaled vector's digits, then the tiles
      const int* rowexp = fx_rowexp();
      launch(fx_split_vector<1024, true>, dim3(1), dim3(1024), x, n, w.xfx2, w.xmeta2, cst, rowexp);
      static const bool opted =
          cudaFuncSetAttribute((const void*)gemv_fx_tile_h, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kFxTileSmem) == cudaSuccess;
      (void)opted;
      launch_smem(gemv_fx_tile_h, grid, dim3(kBlock), kFxTileSmem, A, lda, C, rowexp, n, rpr, x,
                  static_cast<const int4*>(w.xfx2), static_cast<const int*>(w.xmeta2), P2, cst, rec);
    } else {
      launch(gemv_tile_h<R, 1, Dense<R>::E>, grid, dim3(kBlock), A, lda, n, rpr, x, P2, cst, rec);
    }
    timing_end(h, kDt, CCG_SWEEP_C, d.sweep_bytes());
    MvOut<R> m; m.y = nullptr; m.P = w.P2; m.ld = d.n; m.nparts = d.tc.nsplit;
    return m;
  }
  // A x1 and A^H x2: dense operators from one sweep (ncb partials in P1,
  // nsplit in P2); others, and complex128 operators on the integer pipe
  // (whose two sweeps run faster than one fused one), by two applications
  // into y1, y2.
  void apply_both(const cx<R>* x1, const cx<R>* x2, cx<R>* y1, cx<R>* y2, MvOut<R>& o1, MvOut<R>& o2,
                  const SolveState* st) {
    if (op->kind != CCG_OPK_DENSE || fx_digits() != nullptr) {
      o1 = apply_n(x1, y1, st);
      o2 = apply_c(x2, y2, st);
      return;
    }
    dim3 grid(d.ncb, d.tb.nsplit);
    const int64_t rpr = d.tb.rows_per_range;
    timing_begin(h);
    int* rec = timing_rec(h);
    const cx<R>* A = d.A;
    const int64_t lda = d.lda, n = d.n;
    const SolveState* cst = st;
    cx<R>* P1 = w.P1;
    cx<R>* P2 = w.P2;
    if constexpr (sizeof(R) == 4) {
      if (d.unit == 2)
        launch(gemv_tile<R, 2, Dense<R>::E, true, true>, grid, dim3(kBlock), A, lda, n, rpr, x1, x2, P1, P2, cst, rec);
      else
        launch(gemv_tile<R, 1, Dense<R>::E, true, true>, grid, dim3(kBlock), A, lda, n, rpr, x1, x2, P1, P2, cst, rec);
    } else {
      launch(gemv_tile<R, 1, Dense<R>::E, true, true>, grid, dim3(kBlock), A, lda, n, rpr, x1, x2, P1, P2, cst, rec);
    }
    timing_end(h, kDt, CCG_SWEEP_BOTH, d.sweep_bytes());
    o1.y = nullptr; o1.P = w.P1; o1.ld = d.n; o1.nparts = d.ncb;
    o2.y = nullptr; o2.P = w.P2; o2.ld = d.n; o2.nparts = d.tb.nsplit;
  }
};

// Iterations to enqueue between polls: about 50 us of matrix traffic.
template <class R> static int poll_chunk(const Dense<R>& d) {
  const double t_iter = 2.0 * d.sweep_bytes() / 5e12;
  const int c = (int)std::ceil(50e-6 / std::max(t_iter, 1e-9));
  return std::max(1, std::min(c, 4));
}

// Host or device vectors?  Both y and x must be of the same kind.
static int classify(const void* y, const void* x, bool* host) {
  cudaPointerAttributes ay, ax;
  CCG_CUDA(cudaPointerGetAttributes(&ay, y));
  CCG_CUDA(cudaPointerGetAttributes(&ax, x));
  const bool hy = ay.type == cudaMemoryTypeUnregistered || ay.type == cudaMemoryTypeHost;
  const bool hx = ax.type == cudaMemoryTypeUnregistered || ax.type == cudaMemoryTypeHost;
  if (hy != hx) { set_error("y and x must both be host or both be device pointers"); return CCG_ERR_INVALID; }
  *host = hy;
  return CCG_OK;
}

// One solve on device vectors y, x with the workspace w: r0, the method's
// iterations, polling; returns with the stream idle and the final state in
// *fin.  x0_zero skips the A x0 sweep (x is then set to zero on entry).
// A failed operator callback ends the call: read and clear the handle's
// callback status.
static int cb_check(ccg_handle* h) {
  if (h->cb_status == 0) return CCG_OK;
  const int rc = h->cb_status;
  h->cb_status = 0;
  set_error("operator callback returned " + std::to_string(rc));
  return CCG_ERR_CUDA;
}

template <class R>
static int solve_core(ccg_handle* h, int method, const ccg_operator* op, const Ws<R>& w, const cx<R>* y, cx<R>* x,
                      double tol, int maxit, bool x0_zero, SolveState* fin) {
  const int64_t n = op->n;
  Runner<R> run(h, op, w);
  cudaStream_t s = h->stream;

  SolveState init;
  std::memset(&init, 0, sizeof(init));
  init.maxit = maxit;
  init.tol = tol;
  init.hist = w.hist;
  init.skip_mv = x0_zero ? 0 : 1;   // without a known-zero start, the device checks x0
  CCG_CUDA(cudaMemcpyAsync(w.st, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  CCG_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(unsigned int), s));
  if (w.gm.counter) CCG_CUDA(cudaMemsetAsync(w.gm.counter, 0, counter_words(gm_grid(n)) * sizeof(unsigned int), s));
  if (x0_zero) CCG_CUDA(cudaMemsetAsync(x, 0, n * sizeof(cx<R>), s));
  else {
    x_zero_check<R><<<run.grid_vec, kBlock, 0, s>>>(x, n, w.st);
    ++h->launches;
  }

  cx<R>* const* V = w.vec;
  SolveState* st = w.st;

  // r0 = y - A x0
  {
    InitR<R> p;
    p.n = n; p.y = y; p.r = V[0]; p.c1 = nullptr; p.c2 = nullptr; p.method = method;
    switch (method) {
      case M_BICGSTAB: p.c1 = V[1]; break;               // r^
      case M_QMR: p.c1 = V[1]; p.c2 = V[2]; break;       // v~, w~
      case M_COCG: p.c1 = V[1]; break;                   // p
      case M_BICG: p.c1 = V[1]; break;                   // r~
      case M_CGS: p.c1 = V[1]; break;                    // r^
      case M_TFQMR: p.c1 = V[1]; p.c2 = V[2]; break;     // w, u (r itself is r^)
      case M_BICGSTABL: p.c1 = V[2 * kMaxEll + 2]; break; // r~
      default: break;
    }
    if (x0_zero) {
      p.ax.y = nullptr; p.ax.P = nullptr; p.ax.ld = n; p.ax.nparts = 0;
    } else {
      p.ax = run.apply_n(x, V[11], st, false);
    }
    run.phase(p);
  }

  // Per-method vector slots and one iteration's launches.
  std::function<void()> step;
  if (method == M_BICGSTAB) {
    cx<R>*r = V[0], *rh = V[1], *pv = V[2], *v = V[3], *sv = V[4], *t = V[5];
    step = [=, &run]() {
      BiP<R> a; a.n = n; a.r = r; a.p = pv; a.v = v; run.phase(a);
      BiSigma<R> b; b.n = n; b.v = v; b.rh = rh; b.mv = run.apply_n(pv, v, st); run.phase(b);
      BiS<R> c; c.n = n; c.r = r; c.v = v; c.s = sv; run.phase(c);
      BiOmega<R> e; e.n = n; e.t = t; e.s = sv; e.mv = run.apply_n(sv, t, st); run.phase(e);
      BiXR<R> f; f.n = n; f.x = x; f.r = r; f.p = pv; f.s = sv; f.t = t; f.rh = rh; run.phase(f);
    };
  } else if (method == M_CGNR) {
    cx<R>*r = V[0], *z = V[1], *pv = V[2], *wv = V[3];
    CgZ<R> z0; z0.n = n; z0.z = z; z0.p = pv; z0.mv = run.apply_c(r, z, st); run.phase(z0);
    step = [=, &run]() {
      CgAlpha<R> a; a.n = n; a.w = wv; a.mv = run.apply_n(pv, wv, st); run.phase(a);
      CgXR<R> b; b.n = n; b.x = x; b.r = r; b.p = pv; b.w = wv; run.phase(b);
      CgZ<R> c; c.n = n; c.z = z; c.p = nullptr; c.mv = run.apply_c(r, z, st); run.phase(c);
      CgP<R> e; e.n = n; e.z = z; e.p = pv; run.phase(e);
    };
  } else if (method == M_QMR) {
    cx<R>*r = V[0], *vt = V[1], *wt = V[2], *v = V[3], *wv = V[4], *pv = V[5], *q = V[6], *pt = V[7], *u = V[8],
         *dv = V[9], *sv = V[10];
    QVW<R> f; f.n = n; f.vt = vt; f.wt = wt; f.v = v; f.w = wv; run.phase(f);
    step = [=, &run]() {
      QPQ<R> a; a.n = n; a.v = v; a.w = wv; a.p = pv; a.q = q; run.phase(a);
      QEps<R> b; b.n = n; b.pt = pt; b.u = u; b.q = q; run.apply_both(pv, q, pt, u, b.mv1, b.mv2, st); run.phase(b);
      QVT<R> c; c.n = n; c.pt = pt; c.u = u; c.v = v; c.w = wv; c.vt = vt; c.wt = wt; run.phase(c);
      QDX<R> e; e.n = n; e.p = pv; e.pt = pt; e.d = dv; e.s = sv; e.x = x; e.r = r; e.vt = vt; e.wt = wt; e.v = v;
      e.w = wv; run.phase(e);
    };
  } else if (method == M_COCG) {
    cx<R>*r = V[0], *pv = V[1], *q = V[2];
    step = [=, &run]() {
      CoMu<R> a; a.n = n; a.q = q; a.p = pv; a.mv = run.apply_n(pv, q, st); run.phase(a);
      CoXR<R> b; b.n = n; b.x = x; b.r = r; b.p = pv; b.q = q; run.phase(b);
      CoP<R> c; c.n = n; c.r = r; c.p = pv; run.phase(c);
    };
  } else if (method == M_COCR) {
    cx<R>*r = V[0], *pv = V[1], *q = V[2], *wv = V[3];
    auto rho_pq = [=, &run]() {
      CrRho<R> a; a.n = n; a.w = wv; a.r = r; a.mv = run.apply_n(r, wv, st); run.phase(a);
      CrPQ<R> b; b.n = n; b.r = r; b.w = wv; b.p = pv; b.q = q; run.phase(b);
    };
    rho_pq();  // w = A r0, rho, p = r0, q = w, alpha
    step = [=, &run]() {
      CrXR<R> c; c.n = n; c.x = x; c.r = r; c.p = pv; c.q = q; run.phase(c);
      rho_pq();
    };
  } else if (method == M_CGS) {
    cx<R>*r = V[0], *rh = V[1], *u = V[2], *pv = V[3], *q = V[4], *v = V[5], *uh = V[6], *qh = V[7];
    step = [=, &run]() {
      CsUP<R> a; a.n = n; a.r = r; a.q = q; a.u = u; a.p = pv; run.phase(a);
      CsSigma<R> b; b.n = n; b.v = v; b.rh = rh; b.mv = run.apply_n(pv, v, st); run.phase(b);
      CsQ<R> c; c.n = n; c.u = u; c.v = v; c.q = q; c.uh = uh; c.x = x; run.phase(c);
      CsR<R> e; e.n = n; e.r = r; e.rh = rh; e.mv = run.apply_n(uh, qh, st); run.phase(e);
    };
  } else if (method == M_CGNE) {
    cx<R>*r = V[0], *pv = V[1], *wv = V[2], *z = V[3];
    CnP<R> p0; p0.n = n; p0.p = pv; p0.mv = run.apply_c(r, z, st); run.phase(p0);
    step = [=, &run]() {
      CnXR<R> a; a.n = n; a.x = x; a.r = r; a.p = pv; a.mv = run.apply_n(pv, wv, st); run.phase(a);
      CnP<R> b; b.n = n; b.p = pv; b.mv = run.apply_c(r, z, st); run.phase(b);
    };
  } else if (method == M_BICGSTABL) {
    const int L = h->bicgstab_l;
    BlVecs vv;
    for (int i = 0; i <= kMaxEll; ++i) {
      vv.rh[i] = V[i];
      vv.uh[i] = V[kMaxEll + 1 + i];
    }
    const cx<R>* rt = V[2 * kMaxEll + 2];
    { ZeroVec<R> z; z.n = n; z.v = static_cast<cx<R>*>(vv.uh[0]); run.phase(z); }
    { BlRho<R> a; a.n = n; a.mv = run.plain(V[0]); a.out = V[0]; a.rt = rt; a.start = true; run.phase(a); }
    step = [=, &run]() {
      for (int j = 0; j < L; ++j) {
        cx<R>* uj = static_cast<cx<R>*>(vv.uh[j]);
        cx<R>* uj1 = static_cast<cx<R>*>(vv.uh[j + 1]);
        cx<R>* rj = static_cast<cx<R>*>(vv.rh[j]);
        cx<R>* rj1 = static_cast<cx<R>*>(vv.rh[j + 1]);
        BlU<R> a; a.n = n; a.vv = vv; a.j = j; run.phase(a);
        BlGamma<R> b; b.n = n; b.out = uj1; b.rt = rt; b.mv = run.apply_n(uj, uj1, st); run.phase(b);
        BlR<R> c; c.n = n; c.vv = vv; c.j = j; c.x = x; run.phase(c);
        MvOut<R> mv = run.apply_n(rj, rj1, st);
        if (j + 1 < L) {
          BlRho<R> e; e.n = n; e.mv = mv; e.out = rj1; e.rt = rt; e.start = false; run.phase(e);
        } else {
          switch (L) {
            case 1: { BlGram<R, 1> gm; gm.n = n; gm.mv = mv; gm.vv = vv; run.phase(gm); break; }
            case 2: { BlGram<R, 2> gm; gm.n = n; gm.mv = mv; gm.vv = vv; run.phase(gm); break; }
            case 3: { BlGram<R, 3> gm; gm.n = n; gm.mv = mv; gm.vv = vv; run.phase(gm); break; }
            default: { BlGram<R, 4> gm; gm.n = n; gm.mv = mv; gm.vv = vv; run.phase(gm); break; }
          }
        }
      }
      BlMR<R> f; f.n = n; f.vv = vv; f.L = L; f.x = x; f.rt = rt; run.phase(f);
    };
  } else if (method == M_TFQMR) {
    cx<R>*rh = V[0], *wv = V[1], *u = V[2], *un = V[3], *v = V[4], *uh = V[5], *dv = V[6];
    TqInit<R> t0; t0.n = n; t0.v = v; t0.d = dv; run.phase(t0);
    run.apply_n(u, uh, st);  // A u_0
    step = [=, &run]() {
      TqSigma<R> a; a.n = n; a.v = v; a.rh = rh; a.mv = run.plain(uh); run.phase(a);
      TqHalf<R, false> e; e.n = n; e.x = x; e.w = wv; e.d = dv; e.um = u; e.un = un; e.v = v; e.uh = uh; e.rh = rh;
      run.phase(e);
      TqXStop<R> s1; s1.n = n; s1.x = x; s1.d = dv; run.phase(s1);
      run.apply_n(un, uh, st);  // A u_{m+1}
      TqHalf<R, true> o; o.n = n; o.x = x; o.w = wv; o.d = dv; o.um = un; o.un = nullptr; o.v = v; o.uh = uh; o.rh = rh;
      run.phase(o);
      TqXStop<R> s2; s2.n = n; s2.x = x; s2.d = dv; run.phase(s2);
      TqU<R> uu; uu.n = n; uu.w = wv; uu.un = un; uu.uh = uh; uu.u = u; uu.v = v; run.phase(uu);
      run.apply_n(u, uh, st);   // A u for the next iteration
    };
  } else if (method == M_GMRES) {
    if (w.gm.m < 1) {
      set_error("GMRES workspace missing");
      return CCG_ERR_INVALID;
    }
    const int m = w.gm.m;
    cx<R>*r = V[0], *wv = V[1], *t = V[2];
    const Ws<R> ws = w;
    auto begin = [=, &run]() {
      GmBegin<R> b0; b0.n = n; b0.r = r; b0.v0 = ws.basis; b0.b = ws.gm; run.phase(b0);
    };
    begin();
    auto count = std::make_shared<int>(0);
    step = [=, &run]() {
      const int j = *count % m;
      ++*count;
      cx<R>* vj = ws.basis + (int64_t)j * ws.ldv;
      run.apply_n(vj, wv, st);
      run.template gm_pass_launch<GM_DOT>(wv, j);
      run.template gm_pass_launch<GM_UPD_DOT>(wv, j);
      run.template gm_pass_launch<GM_UPD_NORM>(wv, j);
      GmScale<R> sc; sc.n = n; sc.w = wv; sc.v = vj + ws.ldv; run.phase(sc);
      // cycle end (x += V y): at the last step of a cycle, or at once if the
      // cycle stopped early; then the restart
      const bool end = j == m - 1 || *count == maxit;
      gm_solve<<<1, 32, 0, run.s>>>(ws.gm, st, end ? 1 : 0);
      ++run.h->launches;
      GmXUpd<R> xu; xu.n = n; xu.x = x; xu.V = ws.basis; xu.ldv = ws.ldv; xu.yv = ws.gm.yv; xu.always = end;
      run.phase(xu);
      if (end && *count < maxit) {
        GmRestart<R> rs; rs.n = n; rs.y = y; rs.r = r; rs.ax = run.apply_n(x, t, st); run.phase(rs);
        begin();
      }
    };
  } else {  // BiCG
    cx<R>*r = V[0], *rt = V[1], *pv = V[2], *pt = V[3], *q = V[4], *qt = V[5];
    step = [=, &run]() {
      BgP<R> a; a.n = n; a.r = r; a.rt = rt; a.p = pv; a.pt = pt; run.phase(a);
      BgSigma<R> b; b.n = n; b.q = q; b.qt = qt; b.pt = pt; run.apply_both(pv, pt, q, qt, b.mv1, b.mv2, st);
      run.phase(b);
      BgXR<R> c; c.n = n; c.x = x; c.r = r; c.rt = rt; c.p = pv; c.q = q; c.qt = qt; run.phase(c);
    };
  }
  CCG_CUDA(cudaGetLastError());

  // Enqueue iterations in chunks; poll the device record of the chunk before.
  Poll* pin = static_cast<Poll*>(h->pinned);
  const int chunk = poll_chunk(run.d);
  int rc0 = cb_check(h);   // a product enqueued before the loop may have failed
  if (rc0 != CCG_OK) return rc0;
  int launched = 0, npoll = 0;
  for (;;) {
    if (launched < maxit) {
      const int c = std::min(chunk, maxit - launched);
      for (int j = 0; j < c; ++j) step();
      launched += c;
      CCG_CUDA(cudaGetLastError());
      if (h->cb_status) {
        CCG_CUDA(cudaStreamSynchronize(s));
        return cb_check(h);
      }
    }
    const int slot = npoll & 1;
    CCG_CUDA(cudaMemcpyAsync(&pin[slot], &st->poll, sizeof(Poll), cudaMemcpyDeviceToHost, s));
    CCG_CUDA(cudaEventRecord(h->poll_ev[slot], s));
    if (npoll > 0) {
      CCG_CUDA(cudaEventSynchronize(h->poll_ev[slot ^ 1]));
      if (pin[slot ^ 1].done) break;
    }
    ++npoll;
    if (launched >= maxit) break;
  }
  CCG_CUDA(cudaStreamSynchronize(s));
  if ((rc0 = cb_check(h)) != CCG_OK) return rc0;
  CCG_CUDA(cudaMemcpy(fin, st, sizeof(SolveState), cudaMemcpyDeviceToHost));
  if (!fin->poll.done) {  // cannot happen: maxit bounds the loop and the last iteration stops the solve
    set_error("solve did not record its end");
    return CCG_ERR_CUDA;
  }
  return CCG_OK;
}

// A solve on device vectors: one persistent launch where it applies (see
// pk_eligible; `meta` holds pk_meta_bytes(1, dtype) of device memory), else
// the kernel-per-step loop.
template <class R>
static int solve_any(ccg_handle* h, int method, const ccg_operator* op, const Ws<R>& w, const cx<R>* y, cx<R>* x,
                     double tol, int maxit, bool x0_zero, SolveState* fin, char* meta) {
  if (meta != nullptr && pk_eligible(h, method, op)) {
    PkJob<R> j;
    j.op = op; j.w = w; j.y = y; j.x = x; j.tol = tol; j.maxit = maxit; j.x0_zero = x0_zero; j.fin = fin;
    return pk_solve_jobs<R>(h, method, 1, &j, meta);
  }
  return solve_core<R>(h, method, op, w, y, x, tol, maxit, x0_zero, fin);
}

// ||y - A x|| / ||y|| from the final x (one more sweep), with st forced live.
template <class R>
static int true_residual(ccg_handle* h, const ccg_operator* op, const Ws<R>& w, const SolveState& fin,
                         const cx<R>* y, const cx<R>* x, double* out) {
  Runner<R> run(h, op, w);
  SolveState live = fin;
  live.poll.done = 0;
  live.half = 0;
  CCG_CUDA(cudaMemcpyAsync(w.st, &live, sizeof(live), cudaMemcpyHostToDevice, h->stream));
  TrueRes<R> tr;
  tr.n = op->n; tr.y = y; tr.out = w.scratch;
  tr.ax = run.apply_n(x, w.vec[11], w.st);
  run.phase(tr);
  CCG_CUDA(cudaGetLastError());
  if (int rc = cb_check(h)) return rc;
  double rr = 0.0;
  CCG_CUDA(cudaMemcpyAsync(&rr, w.scratch, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CCG_CUDA(cudaStreamSynchronize(h->stream));
  *out = fin.poll.ynorm > 0 ? std::sqrt(rr) / fin.poll.ynorm : 0.0;
  return CCG_OK;
}

template <class R>
static int run_dense(ccg_handle* h, int method, const ccg_operator* op, const void* y_in, void* x_in, double tol,
                     int maxit, double* res_hist, ccg_info* info) {
  const int64_t n = op->n;
  Dense<R> dl(op, h->num_sms);
  const int basis = method == M_GMRES ? h->gm_restart + 1 : 0;
  const size_t wb = ws_bytes<R>(n, dl, maxit, basis);
  int rc = arena_reserve(h, wb + pk_meta_bytes(1, op->dtype));
  if (rc != CCG_OK) return rc;
  Ws<R> w = ws_carve<R>(h->arena, n, dl, maxit, basis);
  char* meta = h->arena + wb;
  cudaStream_t s = h->stream;
  bool host = false;
  if ((rc = classify(y_in, x_in, &host)) != CCG_OK) return rc;
  const cx<R>* y = static_cast<const cx<R>*>(y_in);
  cx<R>* x = static_cast<cx<R>*>(x_in);
  if (host) {
    CCG_CUDA(cudaMemcpyAsync(w.ystage, y_in, n * sizeof(cx<R>), cudaMemcpyHostToDevice, s));
    CCG_CUDA(cudaMemcpyAsync(w.xstage, x_in, n * sizeof(cx<R>), cudaMemcpyHostToDevice, s));
    y = w.ystage;
    x = w.xstage;
  }
  SolveState fin;
  if ((rc = solve_any<R>(h, method, op, w, y, x, tol, maxit, false, &fin, meta)) != CCG_OK) return rc;
  const int iters = fin.poll.k;
  if (fin.zero_rhs) CCG_CUDA(cudaMemsetAsync(x, 0, n * sizeof(cx<R>), s));
  if (res_hist) CCG_CUDA(cudaMemcpyAsync(res_hist, w.hist, (size_t)(iters + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  double true_rel = -1.0;
  if (info && (rc = true_residual<R>(h, op, w, fin, y, x, &true_rel)) != CCG_OK) return rc;
  if (host) CCG_CUDA(cudaMemcpyAsync(x_in, x, n * sizeof(cx<R>), cudaMemcpyDeviceToHost, s));
  CCG_CUDA(cudaStreamSynchronize(s));
  timing_collect(h);
  if (info) {
    info->iters = iters;
    info->status = fin.poll.status;
    info->breakdown = fin.poll.breakdown;
    info->reserved = 0;
    info->relres = fin.poll.relres;
    info->ynorm = fin.poll.ynorm;
    info->true_relres = true_rel;
  }
  return fin.poll.status;
}

int solve_dense(ccg_handle* h, int method, const ccg_operator* op, const void* y, void* x, double tol, int maxit,
                double* res_hist, ccg_info* info) {
  if (op->dtype == CCG_C128) return run_dense<double>(h, method, op, y, x, tol, maxit, res_hist, info);
  return run_dense<float>(h, method, op, y, x, tol, maxit, res_hist, info);
}

// ---------------------------------------------------------------------------
// Mixed-precision iterative refinement: r = y - A x and x += d in complex128,
// the correction A d = r solved by a complex64 Krylov method.
// ---------------------------------------------------------------------------
int solve_refined(ccg_handle* h, int method, const ccg_operator* op, const ccg_operator* op_in, const void* y_in,
                  void* x_in, double tol, int max_outer, double inner_tol, int inner_maxit, double* res_hist,
                  int* inner_iters, ccg_info* info) {
  const int64_t n = op->n;
  Dense<double> d64(op, h->num_sms);
  Dense<float> d32(op_in, h->num_sms);
  const size_t b64 = ws_bytes<double>(n, d64, max_outer);
  const int basis = method == M_GMRES ? h->gm_restart + 1 : 0;
  const size_t b32 = ws_bytes<float>(n, d32, inner_maxit, basis);
  int rc = arena_reserve(h, b64 + b32 + pk_meta_bytes(1, CCG_C64));
  if (rc != CCG_OK) return rc;
  Ws<double> w = ws_carve<double>(h->arena, n, d64, max_outer);
  Ws<float> wi = ws_carve<float>(h->arena + b64, n, d32, inner_maxit, basis);
  char* meta = h->arena + b64 + b32;
  cudaStream_t s = h->stream;
  bool host = false;
  if ((rc = classify(y_in, x_in, &host)) != CCG_OK) return rc;
  const double2* y = static_cast<const double2*>(y_in);
  double2* x = static_cast<double2*>(x_in);
  if (host) {
    CCG_CUDA(cudaMemcpyAsync(w.ystage, y_in, n * sizeof(double2), cudaMemcpyHostToDevice, s));
    CCG_CUDA(cudaMemcpyAsync(w.xstage, x_in, n * sizeof(double2), cudaMemcpyHostToDevice, s));
    y = w.ystage;
    x = w.xstage;
  }
  float2* r32 = wi.ystage;   // right-hand side of the inner solve
  float2* dd = wi.xstage;    // its solution, the correction
  Runner<double> run(h, op, w);

  SolveState init;
  std::memset(&init, 0, sizeof(init));
  init.maxit = max_outer;
  init.tol = tol;
  init.hist = w.hist;
  init.skip_mv = 1;
  CCG_CUDA(cudaMemcpyAsync(w.st, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  CCG_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(unsigned int), s));
  x_zero_check<double><<<run.grid_vec, kBlock, 0, s>>>(x, n, w.st);   // x0 = 0: no first product
  ++h->launches;

  int total_inner = 0, status = CCG_NOT_CONVERGED, bd = 0;
  SolveState outer_state;
  std::memset(&outer_state, 0, sizeof(outer_state));
  for (int outer = 0;; ++outer) {
    RefResid rp;
    rp.n = n; rp.y = y; rp.r32 = r32; rp.d32 = dd; rp.outer = outer;
    rp.ax = run.apply_n(x, w.vec[0], w.st, outer > 0);
    run.phase(rp);
    CCG_CUDA(cudaGetLastError());
    if ((rc = cb_check(h)) != CCG_OK) return rc;
    CCG_CUDA(cudaMemcpyAsync(h->pinned, &w.st->poll, sizeof(Poll), cudaMemcpyDeviceToHost, s));
    CCG_CUDA(cudaStreamSynchronize(s));
    const Poll pl = *static_cast<Poll*>(h->pinned);
    outer_state.poll = pl;
    if (pl.done) { status = pl.status; break; }
    SolveState fin;
    if ((rc = solve_any<float>(h, method, op_in, wi, r32, dd, inner_tol, inner_maxit, true, &fin, meta)) != CCG_OK)
      return rc;
    total_inner += fin.poll.k;
    if (fin.poll.status == ST_NONFINITE) { status = CCG_ERR_NONFINITE; break; }
    if (fin.poll.status == ST_BREAKDOWN && fin.poll.k == 0) { status = CCG_BREAKDOWN; bd = fin.poll.breakdown; break; }
    RefUpdate up;
    up.n = n; up.x = x; up.d32 = dd;
    run.phase(up);
  }
  CCG_CUDA(cudaGetLastError());
  const int outer_steps = outer_state.poll.k;
  SolveState fs;
  CCG_CUDA(cudaMemcpy(&fs, w.st, sizeof(fs), cudaMemcpyDeviceToHost));
  if (fs.zero_rhs) CCG_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), s));
  if (res_hist)
    CCG_CUDA(cudaMemcpyAsync(res_hist, w.hist, (size_t)(outer_steps + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (host) CCG_CUDA(cudaMemcpyAsync(x_in, x, n * sizeof(double2), cudaMemcpyDeviceToHost, s));
  CCG_CUDA(cudaStreamSynchronize(s));
  timing_collect(h);
  if (inner_iters) *inner_iters = total_inner;
  if (info) {
    info->iters = outer_steps;
    info->status = status;
    info->breakdown = bd;
    info->reserved = 0;
    info->relres = outer_state.poll.relres;
    info->ynorm = outer_state.poll.ynorm;
    info->true_relres = outer_state.poll.relres;   // the outer residual is recomputed from x in double
  }
  return status;
}

template <class R> static int matvec_t(ccg_handle* h, const ccg_operator* op, int trans, const void* x_, void* y_) {
  Dense<R> dl(op, h->num_sms);
  int rc = arena_reserve(h, ws_bytes<R>(op->n, dl, 0));
  if (rc != CCG_OK) return rc;
  Ws<R> w = ws_carve<R>(h->arena, op->n, dl, 0);
  Runner<R> run(h, op, w);
  const cx<R>* x = static_cast<const cx<R>*>(x_);
  cx<R>* y = static_cast<cx<R>*>(y_);
  SolveState init;
  std::memset(&init, 0, sizeof(init));
  init.hist = w.hist;
  CCG_CUDA(cudaMemcpyAsync(w.st, &init, sizeof(init), cudaMemcpyHostToDevice, h->stream));
  if (!trans) {
    run.apply_n(x, y, nullptr);
  } else {
    MvOut<R> mv = run.apply_c(x, y, nullptr);
    if (mv.P != nullptr) {
      SumParts<R> p;
      p.n = op->n;
      p.y = y;
      p.mv = mv;
      run.phase(p);
    }
  }
  CCG_CUDA(cudaGetLastError());
  return cb_check(h);
}

int matvec_dense(ccg_handle* h, const ccg_operator* op, int trans, const void* x, void* y) {
  if (op->dtype == CCG_C128) return matvec_t<double>(h, op, trans, x, y);
  return matvec_t<float>(h, op, trans, x, y);
}

template <class R> static int dot_t(ccg_handle* h, int64_t n, const void* u, const void* v, int conj, double* out2) {
  ccg_operator fake;
  fake.n = 1;
  fake.lda = 1;
  Dense<R> dl(&fake, h->num_sms);
  int rc = arena_reserve(h, ws_bytes<R>(1, dl, 0));
  if (rc != CCG_OK) return rc;
  Ws<R> w = ws_carve<R>(h->arena, 1, dl, 0);
  SolveState init;
  std::memset(&init, 0, sizeof(init));
  init.hist = w.hist;
  CCG_CUDA(cudaMemcpyAsync(w.st, &init, sizeof(init), cudaMemcpyHostToDevice, h->stream));
  CCG_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(unsigned int), h->stream));
  DotPhase<R> p;
  p.n = n;
  p.u = static_cast<const cx<R>*>(u);
  p.v = static_cast<const cx<R>*>(v);
  p.conj = conj;
  p.out = w.scratch;
  Red red;
  red.partials = w.partials;
  red.counter = w.counter;
  int grid = (int)std::min<int64_t>((n + kBlock - 1) / kBlock, (int64_t)h->num_sms * 8);
  grid = std::max(1, std::min(grid, kMaxRedBlocks));
  phase_kernel<DotPhase<R>, double><<<grid, kBlock, 0, h->stream>>>(p, w.st, red);  // the API dot: double
  ++h->launches;
  CCG_CUDA(cudaGetLastError());
  CCG_CUDA(cudaMemcpyAsync(out2, w.scratch, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CCG_CUDA(cudaStreamSynchronize(h->stream));
  return CCG_OK;
}

int dot_device(ccg_handle* h, ccg_dtype dtype, int64_t n, const void* u, const void* v, int conj, double* out2) {
  if (dtype == CCG_C128) return dot_t<double>(h, n, u, v, conj, out2);
  return dot_t<float>(h, n, u, v, conj, out2);
}

}  // namespace ccg
