// Many right-hand sides at once: A X = Y for k <= 256 columns advancing
// together (the multi-right-hand-side form of the manual's Sec. 1 problem),
// with BiCGSTAB (Sec. 2.1) run independently per column: every column has
// its own scalars, iteration count and stopping test; a stopped column is
// frozen while the others continue.  Per iteration the two operator
// applications are block products A P, A S (blockmv.cuh), so the matrix
// streams once per product for all columns.
//
// Blocks are row-major inside the library (row i holds unknown i of all k
// columns), so a phase kernel gives each column to one thread and splits the
// rows over the grid: loads are coalesced across columns and every column's
// dot products reduce in a fixed order (per block, then over blocks in the
// last block to finish), exactly as the single-right-hand-side phases do.
//
// Mixed precision: complex128 block residuals R = Y - A X and updates
// X += D around complex64 batched inner solves A D = R.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "blockmv.cuh"
#include "common.cuh"
#include "reduce.cuh"
#include "internal.h"

namespace ccg {

struct BCtl {
  int all_done;  // every column has stopped
  int skip_mv;   // the block product's input is zero: skip it
  int maxit;
  int pad;
  double tol;
};

struct BCols {                // per-column state, arrays of k
  double2* rho;
  double2* alpha;
  double2* omega;
  double2* beta;
  double* ynorm;
  double* snorm;
  double* relres;
  int* iters;
  int* status;
  int* bd;
  int* half;
  int* done;
  int* zero_rhs;
  const int* skip;            // optional: columns that start stopped
  double* hist;               // [k][hist_ld]
  int hist_ld;
};


template <class R> using BAcc = acc_t<R>;

struct BPhaseBase {
  using Acc = double;
  static constexpr bool kReduce = true;
  static constexpr bool kCheckAll = false;
  __device__ __forceinline__ bool active(int c, const BCols& s) const { return !s.done[c]; }
};

// Rows whose operands one thread loads before it applies them.
constexpr int kRowsIn = 4;

template <class P>
__global__ void __launch_bounds__(kBlock) bphase_kernel(P p, BCtl* ctl, BCols cols, Red red) {
  if (ctl->all_done) return;
  const int k = p.k;
  const int rpar = kBlock / k;
  const int c = threadIdx.x % k, rs = threadIdx.x / k;
  typename P::Acc acc[P::NQ];
#pragma unroll
  for (int q = 0; q < P::NQ; ++q) acc_zero(acc[q]);
  if (rs < rpar && p.active(c, cols)) {
    typename P::Col cs = p.col(c, cols);
    // kRowsIn rows' operands are loaded before any of them is applied (no
    // phase writes an element another row reads), then applied in row
    // order, so each thread's sums keep the one-row-at-a-time order
    const int64_t stride = (int64_t)gridDim.x * rpar;
    int64_t row = (int64_t)blockIdx.x * rpar + rs;
    for (; row + (kRowsIn - 1) * stride < p.n; row += kRowsIn * stride) {
      typename P::In in[kRowsIn];
#pragma unroll
      for (int u = 0; u < kRowsIn; ++u) in[u] = p.load((row + u * stride) * k + c, cs);
#pragma unroll
      for (int u = 0; u < kRowsIn; ++u) p.apply((row + u * stride) * k + c, cs, in[u], acc);
    }
    for (; row < p.n; row += stride) p.apply(row * k + c, cs, p.load(row * k + c, cs), acc);
  }
  if (!P::kReduce) return;
  __shared__ double sred[P::NQ][kBlock];
  __shared__ bool is_last;
#pragma unroll
  for (int q = 0; q < P::NQ; ++q) sred[q][threadIdx.x] = acc_value(acc[q]);
  __syncthreads();
  auto slot = [&](int b, int q) { return &red.partials[((int64_t)b * P::NQ + q) * k + threadIdx.x]; };
  if (threadIdx.x < k) {
#pragma unroll
    for (int q = 0; q < P::NQ; ++q) {
      double v = 0.0;
      for (int r = 0; r < rpar; ++r) v += sred[q][r * k + threadIdx.x];
      *slot(blockIdx.x, q) = v;
    }
    __threadfence();
  }
  // Deterministic tree reduction with fan-in kRedGroup: at each level the
  // last block of a group sums the group's slots (all loads in flight at
  // once) into the group's first slot and moves up; the block that sums the
  // last remaining group holds the total in slot 0.  Each column's thread
  // walks a fixed order, so results do not depend on which blocks finish
  // last.
  int idx = blockIdx.x, cnt = gridDim.x, stride = 1, base = 0;
  while (cnt > 1) {
    const int g = idx / kRedGroup, g0 = g * kRedGroup;
    const int gsize = min(kRedGroup, cnt - g0);
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned int t = atomicAdd(&red.counter[base + g], 1u);
      is_last = (t == (unsigned)gsize - 1u);
      if (is_last) red.counter[base + g] = 0u;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x < k) {
      double v[kRedGroup][P::NQ];
#pragma unroll
      for (int b = 0; b < kRedGroup; ++b)
#pragma unroll
        for (int q = 0; q < P::NQ; ++q) v[b][q] = b < gsize ? __ldcg(slot((g0 + b) * stride, q)) : 0.0;
#pragma unroll
      for (int q = 0; q < P::NQ; ++q) {
        double t = 0.0;
#pragma unroll
        for (int b = 0; b < kRedGroup; ++b) t += v[b][q];
        *slot(g0 * stride, q) = t;
      }
      __threadfence();
    }
    base += (cnt + kRedGroup - 1) / kRedGroup;
    idx = g;
    cnt = (cnt + kRedGroup - 1) / kRedGroup;
    stride *= kRedGroup;
  }
  __syncthreads();
  if (threadIdx.x < k && !cols.done[threadIdx.x]) {
    double tot[P::NQ];
#pragma unroll
    for (int q = 0; q < P::NQ; ++q) tot[q] = __ldcg(slot(0, q));
    p.finish(threadIdx.x, tot, cols, ctl);
  }
  __syncthreads();
  if (P::kCheckAll) {
    const int nd = __syncthreads_count(threadIdx.x < k && cols.done[threadIdx.x]);
    if (threadIdx.x == 0 && nd == k) ctl->all_done = 1;
  }
}

template <class T> __device__ __forceinline__ void b_dotc(double* acc, T u, T v) {
  const double2 a = widen(u), b = widen(v);
  acc[0] += a.x * b.x + a.y * b.y;
  acc[1] += a.x * b.y - a.y * b.x;
}
template <class T> __device__ __forceinline__ void b_nrm2(double* acc, T u) {
  const double2 a = widen(u);
  acc[0] += a.x * a.x + a.y * a.y;
}
__device__ __forceinline__ void b_dotc(FF* acc, float2 a, float2 b) {
  ff_add_prod(acc[0], a.x, b.x);
  ff_add_prod(acc[0], a.y, b.y);
  ff_add_prod(acc[1], a.x, b.y);
  ff_add_prod(acc[1], -a.y, b.x);
}
__device__ __forceinline__ void b_nrm2(FF* acc, float2 a) {
  ff_add_prod(acc[0], a.x, a.x);
  ff_add_prod(acc[0], a.y, a.y);
}
template <class R> __device__ __forceinline__ bool b_tiny(double2 s) { return cabs(s) < tiny_guard<R>(); }
template <class R> __device__ __forceinline__ bool b_tiny(double s) { return fabs(s) < tiny_guard<R>(); }
__device__ __forceinline__ bool b_nonfinite(double v) { return !(v == v) || isinf(v); }

__device__ __forceinline__ void col_stop(const BCols& s, int c, int status, int bd) {
  s.status[c] = status;
  s.bd[c] = bd;
  s.done[c] = 1;
}
// End of iteration it of column c: converged, breakdown, cap (the
// single-right-hand-side order).  Returns true if the column stops.
__device__ __forceinline__ bool col_end(const BCols& s, const BCtl* ctl, int c, int it, double rel, int bd) {
  s.iters[c] = it;
  s.relres[c] = rel;
  s.hist[(int64_t)c * s.hist_ld + it] = rel;
  if (b_nonfinite(rel)) { col_stop(s, c, ST_NONFINITE, 0); return true; }
  if (rel <= ctl->tol) { col_stop(s, c, ST_OK, 0); return true; }
  if (bd) { col_stop(s, c, ST_BREAKDOWN, bd); return true; }
  if (it >= ctl->maxit) { col_stop(s, c, ST_NOT_CONVERGED, 0); return true; }
  return false;
}

// R = Y - A X0 (ax null: X0 = 0), R^ = R; per-column ||y||, ||r||, start scalars.
template <class R> struct BInit : BPhaseBase {
  using Acc = BAcc<R>;
  static constexpr int NQ = 3;
  static constexpr bool kCheckAll = true;
  struct Col {};
  int64_t n;
  int k;
  const cx<R>* y;
  const cx<R>* ax;
  cx<R>* r;
  cx<R>* rh;
  __device__ __forceinline__ bool active(int c, const BCols& s) const { return !s.done[c] && !(s.skip && s.skip[c]); }
  __device__ __forceinline__ Col col(int, const BCols&) const { return Col(); }
  struct In { cx<R> y, ax; };
  __device__ __forceinline__ In load(int64_t e, const Col&) const {
    In in;
    in.y = y[e];
    in.ax = ax ? ax[e] : mk<R>(0, 0);
    return in;
  }
  __device__ __forceinline__ void apply(int64_t e, const Col&, const In& in, Acc* acc) const {
    const cx<R> yi = in.y;
    const cx<R> ri = ax ? csub(yi, in.ax) : yi;
    r[e] = ri;
    rh[e] = ri;
    b_nrm2(acc, yi);
    b_nrm2(acc + 1, ri);
    if (!(isfinite((double)yi.x) && isfinite((double)yi.y))) acc_add1(acc[2]);
  }
  __device__ void finish(int c, const double* t, const BCols& s, const BCtl* ctl) const {
    s.iters[c] = 0;
    if (s.skip && s.skip[c]) { s.relres[c] = 0.0; s.hist[(int64_t)c * s.hist_ld] = 0.0; col_stop(s, c, ST_OK, 0); return; }
    if (t[2] != 0.0) { col_stop(s, c, ST_NONFINITE, 0); return; }
    const double yn = sqrt(t[0]);
    s.ynorm[c] = yn;
    if (yn == 0.0) {
      s.zero_rhs[c] = 1;
      s.relres[c] = 0.0;
      s.hist[(int64_t)c * s.hist_ld] = 0.0;
      col_stop(s, c, ST_OK, 0);
      return;
    }
    const double rel = sqrt(t[1]) / yn;
    s.relres[c] = rel;
    s.hist[(int64_t)c * s.hist_ld] = rel;
    if (b_nonfinite(rel)) { col_stop(s, c, ST_NONFINITE, 0); return; }
    if (rel <= ctl->tol) { col_stop(s, c, ST_OK, 0); return; }
    if (ctl->maxit <= 0) { col_stop(s, c, ST_NOT_CONVERGED, 0); return; }
    s.rho[c] = mkc(t[1], 0.0);
    s.alpha[c] = s.omega[c] = mkc(1.0, 0.0);
    if (b_tiny<R>(s.rho[c])) col_stop(s, c, ST_BREAKDOWN, CCG_BD_RHO);
  }
};

template <class R> struct BP : BPhaseBase {  // p = r (first) or r + beta (p - omega v)
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  struct Col { cx<R> beta, omega; bool first; };
  int64_t n;
  int k;
  const cx<R>* r;
  cx<R>* p;
  const cx<R>* v;
  __device__ __forceinline__ Col col(int c, const BCols& s) const {
    Col o;
    o.first = s.iters[c] == 0;
    o.beta = narrow<R>(s.beta[c]);
    o.omega = narrow<R>(s.omega[c]);
    return o;
  }
  struct In { cx<R> r, p, v; };
  __device__ __forceinline__ In load(int64_t e, const Col& o) const {
    In in;
    in.r = r[e];
    in.p = o.first ? mk<R>(0, 0) : p[e];
    in.v = o.first ? mk<R>(0, 0) : v[e];
    return in;
  }
  __device__ __forceinline__ void apply(int64_t e, const Col& o, const In& in, double*) const {
    p[e] = o.first ? in.r : cadd(in.r, cmul(o.beta, csub(in.p, cmul(o.omega, in.v))));
  }
  __device__ void finish(int, const double*, const BCols&, const BCtl*) const {}
};

template <class R> struct BSigma : BPhaseBase {  // alpha = rho / <r^, v>
  using Acc = BAcc<R>;
  static constexpr int NQ = 2;
  struct Col {};
  int64_t n;
  int k;
  const cx<R>* rh;
  const cx<R>* v;
  __device__ __forceinline__ Col col(int, const BCols&) const { return Col(); }
  struct In { cx<R> rh, v; };
  __device__ __forceinline__ In load(int64_t e, const Col&) const { return In{rh[e], v[e]}; }
  __device__ __forceinline__ void apply(int64_t, const Col&, const In& in, Acc* acc) const { b_dotc(acc, in.rh, in.v); }
  __device__ void finish(int c, const double* t, const BCols& s, const BCtl*) const {
    const double2 sigma = mkc(t[0], t[1]);
    if (b_tiny<R>(sigma)) { col_stop(s, c, ST_BREAKDOWN, CCG_BD_SIGMA); return; }
    s.alpha[c] = cdiv(s.rho[c], sigma);
  }
};

template <class R> struct BS : BPhaseBase {  // s = r - alpha v; half-step exit test on ||s||
  using Acc = BAcc<R>;
  static constexpr int NQ = 1;
  struct Col { cx<R> alpha; };
  int64_t n;
  int k;
  const cx<R>* r;
  const cx<R>* v;
  cx<R>* sv;
  __device__ __forceinline__ Col col(int c, const BCols& s) const { Col o; o.alpha = narrow<R>(s.alpha[c]); return o; }
  struct In { cx<R> r, v; };
  __device__ __forceinline__ In load(int64_t e, const Col&) const { return In{r[e], v[e]}; }
  __device__ __forceinline__ void apply(int64_t e, const Col& o, const In& in, Acc* acc) const {
    const cx<R> si = csub(in.r, cmul(o.alpha, in.v));
    sv[e] = si;
    b_nrm2(acc, si);
  }
  __device__ void finish(int c, const double* t, const BCols& s, const BCtl* ctl) const {
    s.snorm[c] = sqrt(t[0]) / s.ynorm[c];
    s.half[c] = s.snorm[c] <= ctl->tol ? 1 : 0;
  }
};

template <class R> struct BOmega : BPhaseBase {  // omega = <t, s> / <t, t>
  using Acc = BAcc<R>;
  static constexpr int NQ = 3;
  struct Col {};
  int64_t n;
  int k;
  const cx<R>* t;
  const cx<R>* sv;
  __device__ __forceinline__ bool active(int c, const BCols& s) const { return !s.done[c] && !s.half[c]; }
  __device__ __forceinline__ Col col(int, const BCols&) const { return Col(); }
  struct In { cx<R> t, s; };
  __device__ __forceinline__ In load(int64_t e, const Col&) const { return In{t[e], sv[e]}; }
  __device__ __forceinline__ void apply(int64_t, const Col&, const In& in, Acc* acc) const {
    b_dotc(acc, in.t, in.s);
    b_nrm2(acc + 2, in.t);
  }
  __device__ void finish(int c, const double* q, const BCols& s, const BCtl*) const {
    if (s.half[c]) return;
    const double tt = q[2];
    if (b_tiny<R>(tt)) { col_stop(s, c, ST_BREAKDOWN, CCG_BD_TT); return; }
    s.omega[c] = mkc(q[0] / tt, q[1] / tt);
  }
};

template <class R> struct BXR : BPhaseBase {  // x += alpha p + omega s; r = s - omega t; next rho
  using Acc = BAcc<R>;
  static constexpr int NQ = 3;
  static constexpr bool kCheckAll = true;
  struct Col { cx<R> alpha, omega; bool half; };
  int64_t n;
  int k;
  cx<R>* x;
  cx<R>* r;
  const cx<R>* p;
  const cx<R>* sv;
  const cx<R>* t;
  const cx<R>* rh;
  __device__ __forceinline__ Col col(int c, const BCols& s) const {
    Col o;
    o.alpha = narrow<R>(s.alpha[c]);
    o.omega = narrow<R>(s.omega[c]);
    o.half = s.half[c] != 0;
    return o;
  }
  struct In { cx<R> x, p, s, t, rh; };
  __device__ __forceinline__ In load(int64_t e, const Col& o) const {
    In in;
    in.x = x[e];
    in.p = p[e];
    const cx<R> z = mk<R>(0, 0);
    in.s = o.half ? z : sv[e];
    in.t = o.half ? z : t[e];
    in.rh = o.half ? z : rh[e];
    return in;
  }
  __device__ __forceinline__ void apply(int64_t e, const Col& o, const In& in, Acc* acc) const {
    if (o.half) {
      x[e] = cadd(in.x, cmul(o.alpha, in.p));
      return;
    }
    x[e] = cadd(in.x, cadd(cmul(o.alpha, in.p), cmul(o.omega, in.s)));
    const cx<R> ri = csub(in.s, cmul(o.omega, in.t));
    r[e] = ri;
    b_dotc(acc, in.rh, ri);
    b_nrm2(acc + 2, ri);
  }
  __device__ void finish(int c, const double* q, const BCols& s, const BCtl* ctl) const {
    const int it = s.iters[c] + 1;
    if (s.half[c]) {
      s.iters[c] = it;
      s.relres[c] = s.snorm[c];
      s.hist[(int64_t)c * s.hist_ld + it] = s.snorm[c];
      col_stop(s, c, ST_OK, 0);
      return;
    }
    const double rel = sqrt(q[2]) / s.ynorm[c];
    if (col_end(s, ctl, c, it, rel, b_tiny<R>(s.omega[c]) ? CCG_BD_OMEGA : 0)) return;
    const double2 rho_new = mkc(q[0], q[1]);
    if (b_tiny<R>(rho_new)) { col_stop(s, c, ST_BREAKDOWN, CCG_BD_RHO); return; }
    s.beta[c] = cmul(cdiv(rho_new, s.rho[c]), cdiv(s.alpha[c], s.omega[c]));
    s.rho[c] = rho_new;
  }
};

// Outer (complex128) refinement phases.
struct BRefResid : BPhaseBase {  // r32 = round(y - A x), d32 = 0; outer residual per column
  static constexpr int NQ = 3;
  static constexpr bool kCheckAll = true;
  struct Col {};
  int64_t n;
  int k;
  const double2* y;
  const double2* ax;   // null: x = 0
  float2* r32;
  float2* d32;
  int outer;
  __device__ __forceinline__ Col col(int, const BCols&) const { return Col(); }
  struct In { double2 y, ax; };
  __device__ __forceinline__ In load(int64_t e, const Col&) const {
    In in;
    in.y = y[e];
    in.ax = ax ? ax[e] : make_double2(0.0, 0.0);
    return in;
  }
  __device__ __forceinline__ void apply(int64_t e, const Col&, const In& in, double* acc) const {
    const double2 yi = in.y;
    const double2 ri = ax ? csub(yi, in.ax) : yi;
    r32[e] = make_float2((float)ri.x, (float)ri.y);
    d32[e] = make_float2(0.f, 0.f);
    acc[0] += yi.x * yi.x + yi.y * yi.y;
    acc[1] += ri.x * ri.x + ri.y * ri.y;
    if (!(isfinite(yi.x) && isfinite(yi.y))) acc[2] += 1.0;
  }
  __device__ void finish(int c, const double* t, const BCols& s, const BCtl* ctl) const {
    s.iters[c] = outer;
    if (t[2] != 0.0) { col_stop(s, c, ST_NONFINITE, 0); return; }
    const double yn = sqrt(t[0]);
    s.ynorm[c] = yn;
    if (yn == 0.0) {
      s.zero_rhs[c] = 1;
      s.relres[c] = 0.0;
      s.hist[(int64_t)c * s.hist_ld + outer] = 0.0;
      col_stop(s, c, ST_OK, 0);
      return;
    }
    const double rel = sqrt(t[1]) / yn;
    s.relres[c] = rel;
    s.hist[(int64_t)c * s.hist_ld + outer] = rel;
    if (b_nonfinite(rel)) { col_stop(s, c, ST_NONFINITE, 0); return; }
    if (rel <= ctl->tol) { col_stop(s, c, ST_OK, 0); return; }
    if (outer >= ctl->maxit) col_stop(s, c, ST_NOT_CONVERGED, 0);
  }
};
struct BRefUpdate : BPhaseBase {  // x += widen(d32) for columns still refining
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  struct Col {};
  int64_t n;
  int k;
  double2* x;
  const float2* d32;
  __device__ __forceinline__ Col col(int, const BCols&) const { return Col(); }
  struct In { double2 x; float2 d; };
  __device__ __forceinline__ In load(int64_t e, const Col&) const { return In{x[e], d32[e]}; }
  __device__ __forceinline__ void apply(int64_t e, const Col&, const In& in, double*) const {
    x[e] = cadd(in.x, make_double2((double)in.d.x, (double)in.d.y));
  }
  __device__ void finish(int, const double*, const BCols&, const BCtl*) const {}
};

struct BMidResid : BPhaseBase {  // rm = r - A d (complex64, exact product)
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  struct Col {};
  int64_t n;
  int k;
  const float2* r;
  const float2* ad;
  float2* rm;
  __device__ __forceinline__ Col col(int, const BCols&) const { return Col(); }
  struct In { float2 r, ad; };
  __device__ __forceinline__ In load(int64_t e, const Col&) const { return In{r[e], ad[e]}; }
  __device__ __forceinline__ void apply(int64_t e, const Col&, const In& in, double*) const { rm[e] = csub(in.r, in.ad); }
  __device__ void finish(int, const double*, const BCols&, const BCtl*) const {}
};
struct BMidAdd : BPhaseBase {  // d += e
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  struct Col {};
  int64_t n;
  int k;
  float2* d;
  const float2* e;
  __device__ __forceinline__ Col col(int, const BCols&) const { return Col(); }
  struct In { float2 d, e; };
  __device__ __forceinline__ In load(int64_t i, const Col&) const { return In{d[i], e[i]}; }
  __device__ __forceinline__ void apply(int64_t i, const Col&, const In& in, double*) const { d[i] = cadd(in.d, in.e); }
  __device__ void finish(int, const double*, const BCols&, const BCtl*) const {}
};

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
#define B_CUDA(call)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                   \
      return CCG_ERR_CUDA;                                                             \
    }                                                                                  \
  } while (0)

static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

// Device arena carving for one batched solve in precision R.
template <class R> struct BWs {
  cx<R>* vec[8];   // r, r^, p, v, s, t, and two staging blocks
  double* partials;
  unsigned int* counter;  // the reduction's counters: all groups, then one per group
  size_t counter_bytes = 0;
  BCtl* ctl;
  BCols cols;
  static size_t bytes(int64_t n, int k, int maxit, int grid) {
    size_t b = 8 * al256((size_t)n * k * sizeof(cx<R>));
    b += al256((size_t)grid * 4 * k * sizeof(double));
    b += al256(counter_words(grid) * sizeof(unsigned int)) + al256(sizeof(BCtl));
    b += 5 * al256(k * sizeof(double2)) + 3 * al256(k * sizeof(double)) + 6 * al256(k * sizeof(int));
    b += al256((size_t)k * (maxit + 1) * sizeof(double));
    return b;
  }
  void carve(char* base, int64_t n, int k, int maxit, int grid) {
    size_t off = 0;
    auto take = [&](size_t nb) { char* p = base + off; off += al256(nb); return p; };
    for (int i = 0; i < 8; ++i) vec[i] = reinterpret_cast<cx<R>*>(take((size_t)n * k * sizeof(cx<R>)));
    partials = reinterpret_cast<double*>(take((size_t)grid * 4 * k * sizeof(double)));
    counter = reinterpret_cast<unsigned int*>(take(counter_words(grid) * sizeof(unsigned int)));
    counter_bytes = counter_words(grid) * sizeof(unsigned int);
    ctl = reinterpret_cast<BCtl*>(take(sizeof(BCtl)));
    double2** c2[5] = {&cols.rho, &cols.alpha, &cols.omega, &cols.beta, nullptr};
    for (int i = 0; i < 4; ++i) *c2[i] = reinterpret_cast<double2*>(take(k * sizeof(double2)));
    take(k * sizeof(double2));
    cols.ynorm = reinterpret_cast<double*>(take(k * sizeof(double)));
    cols.snorm = reinterpret_cast<double*>(take(k * sizeof(double)));
    cols.relres = reinterpret_cast<double*>(take(k * sizeof(double)));
    int** ci[6] = {&cols.iters, &cols.status, &cols.bd, &cols.half, &cols.done, &cols.zero_rhs};
    for (int i = 0; i < 6; ++i) *ci[i] = reinterpret_cast<int*>(take(k * sizeof(int)));
    cols.hist = reinterpret_cast<double*>(take((size_t)k * (maxit + 1) * sizeof(double)));
    cols.hist_ld = maxit + 1;
    cols.skip = nullptr;
  }
};

static int phase_grid(const ccg_handle* h, int64_t n, int k) {
  const int rpar = kBlock / k;
  const int64_t want = (n + rpar - 1) / rpar;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)h->num_sms * 4));
}

template <class R> struct BRun {
  ccg_handle* h;
  const ccg_operator* op;
  bool allow_tc = false;  // complex64 products may use the tensor cores
  cudaStream_t s;
  int64_t n;
  int k;
  int grid;
  BWs<R> w;
  Red red;

  // A phase runs on at most its resident blocks (one wave: the rows a
  // thread loads ahead need registers, so heavier phases fit fewer blocks);
  // the reduction's slots and counters are sized for `grid`, the largest.
  template <class P> void phase(const P& p) {
    static const int occ = [] {
      int o = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, bphase_kernel<P>, kBlock, 0) != cudaSuccess) {
        cudaGetLastError();
        o = 1;
      }
      return o < 1 ? 1 : o;
    }();
    const int g = (int)std::min<int64_t>(grid, (int64_t)h->num_sms * occ);
    bphase_kernel<P><<<g, kBlock, 0, s>>>(p, w.ctl, w.cols, red);
    ++h->launches;
  }
  // C = A B.  complex64 products go to the split-bf16 tensor-core product
  // when allowed (fast, ~1e-4 accurate); otherwise both precisions go to the
  // exact integer-slice product (as accurate as a GEMM in their own
  // precision) when enabled, else to the CUDA cores.
  int gemm(const cx<R>* B, cx<R>* C, const int* skip) {
    timing_begin(h);
    const int dt = sizeof(R) == 8 ? CCG_C128 : CCG_C64;
    if constexpr (sizeof(R) == 4) {
      if (allow_tc && tc_available(op)) {
        const int rc = tc_block_product(h, op, B, C, k, skip);
        timing_end(h, CCG_C64, CCG_SWEEP_BLOCK_TC, (double)n * n * 8.0 + 2.0 * n * k * sizeof(cx<R>));
        return rc;
      }
    }
    if (h->tc_exact && oz_available(op)) {
      const int rc = oz_block_product(h, op, B, C, k, skip);
      timing_end(h, dt, CCG_SWEEP_BLOCK_EXACT, (double)n * n * sizeof(cx<R>) + 2.0 * n * k * sizeof(cx<R>));
      return rc;
    }
    dim3 g((k + gemm_bn<R>() - 1) / gemm_bn<R>(), (unsigned)((n + gemm_bm<R>() - 1) / gemm_bm<R>()));
    cgemm_rows<R><<<g, kBlock, 0, s>>>(static_cast<const cx<R>*>(op->A), op->lda, B, C, n, k, skip, timing_rec(h));
    ++h->launches;
    timing_end(h, sizeof(R) == 8 ? CCG_C128 : CCG_C64, CCG_SWEEP_BLOCK,
               (double)n * n * sizeof(cx<R>) + 2.0 * n * k * sizeof(cx<R>));
    return CCG_OK;
  }
};

// Batched BiCGSTAB on row-major device blocks Y (input) and X (start in,
// solution out).  x0_zero: X is zero on entry (the first product is
// skipped).  skip: optional device mask of columns that start stopped.
template <class R>
static int bicgstab_core(BRun<R>& run, const cx<R>* Y, cx<R>* X, double tol, int maxit, bool x0_zero,
                         const int* skip) {
  ccg_handle* h = run.h;
  cudaStream_t s = run.s;
  const int64_t n = run.n;
  const int k = run.k;
  BWs<R>& w = run.w;
  BCtl init;
  std::memset(&init, 0, sizeof(init));
  init.maxit = maxit;
  init.tol = tol;
  B_CUDA(cudaMemcpyAsync(w.ctl, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  B_CUDA(cudaMemsetAsync(w.counter, 0, w.counter_bytes, s));
  B_CUDA(cudaMemsetAsync(w.cols.done, 0, k * sizeof(int), s));
  B_CUDA(cudaMemsetAsync(w.cols.half, 0, k * sizeof(int), s));
  B_CUDA(cudaMemsetAsync(w.cols.zero_rhs, 0, k * sizeof(int), s));
  B_CUDA(cudaMemsetAsync(w.cols.iters, 0, k * sizeof(int), s));
  B_CUDA(cudaMemsetAsync(w.cols.status, 0, k * sizeof(int), s));
  B_CUDA(cudaMemsetAsync(w.cols.bd, 0, k * sizeof(int), s));
  w.cols.skip = skip;
  cx<R>*r = w.vec[0], *rh = w.vec[1], *p = w.vec[2], *v = w.vec[3], *sv = w.vec[4], *t = w.vec[5];
  {
    BInit<R> a;
    a.n = n; a.k = k; a.y = Y; a.r = r; a.rh = rh; a.ax = nullptr;
    if (x0_zero) {
      B_CUDA(cudaMemsetAsync(X, 0, (size_t)n * k * sizeof(cx<R>), s));
    } else {
      run.gemm(X, t, nullptr);
      a.ax = t;
    }
    run.phase(a);
  }
  w.cols.skip = nullptr;
  const int* all_done = &w.ctl->all_done;
  auto step = [&]() {
    BP<R> a; a.n = n; a.k = k; a.r = r; a.p = p; a.v = v; run.phase(a);
    run.gemm(p, v, all_done);
    BSigma<R> b; b.n = n; b.k = k; b.rh = rh; b.v = v; run.phase(b);
    BS<R> c; c.n = n; c.k = k; c.r = r; c.v = v; c.sv = sv; run.phase(c);
    run.gemm(sv, t, all_done);
    BOmega<R> d; d.n = n; d.k = k; d.t = t; d.sv = sv; run.phase(d);
    BXR<R> e; e.n = n; e.k = k; e.x = X; e.r = r; e.p = p; e.sv = sv; e.t = t; e.rh = rh; run.phase(e);
  };
  B_CUDA(cudaGetLastError());
  int* pin = static_cast<int*>(h->pinned);
  int launched = 0, npoll = 0;
  for (;;) {
    if (launched < maxit) {
      step();
      ++launched;
      B_CUDA(cudaGetLastError());
    }
    const int slot = npoll & 1;
    B_CUDA(cudaMemcpyAsync(&pin[slot], all_done, sizeof(int), cudaMemcpyDeviceToHost, s));
    B_CUDA(cudaEventRecord(h->poll_ev[slot], s));
    if (npoll > 0) {
      B_CUDA(cudaEventSynchronize(h->poll_ev[slot ^ 1]));
      if (pin[slot ^ 1]) break;
    }
    ++npoll;
    if (launched >= maxit) break;
  }
  B_CUDA(cudaStreamSynchronize(s));
  return CCG_OK;
}

template <class R> __global__ void zero_cols(cx<R>* X, int64_t n, int k, const int* zero) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x)
    if (zero[e % k]) X[e] = mk<R>(0, 0);
}

static void copy_cols_out(const BCols& c, int k, int32_t* iters, int32_t* status, double* relres, cudaStream_t s) {
  if (iters) cudaMemcpyAsync(iters, c.iters, k * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (status) cudaMemcpyAsync(status, c.status, k * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (relres) cudaMemcpyAsync(relres, c.relres, k * sizeof(double), cudaMemcpyDeviceToHost, s);
}

static int worst_status(const std::vector<int>& st) {
  int w = CCG_OK;
  for (int v : st) {
    if (v < 0) return v;
    if (v > w) w = v;
  }
  return w;
}

template <class R>
static int batched_t(ccg_handle* h, const ccg_operator* op, int64_t k, const void* Y, int64_t ldy, void* X,
                     int64_t ldx, double tol, int maxit, int32_t* iters, int32_t* status, double* relres) {
  const int64_t n = op->n;
  const int kk = (int)k;
  BRun<R> run;
  run.h = h; run.op = op; run.s = h->stream; run.n = n; run.k = kk; run.grid = phase_grid(h, n, kk);
  run.allow_tc = h->tc_mode >= 2;
  int rc = arena_reserve(h, BWs<R>::bytes(n, kk, maxit, run.grid));
  if (rc != CCG_OK) return rc;
  run.w.carve(h->arena, n, kk, maxit, run.grid);
  run.red.partials = run.w.partials;
  run.red.counter = run.w.counter;
  cx<R>* Yr = run.w.vec[6];
  cx<R>* Xr = run.w.vec[7];
  dim3 tg((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32));
  block_to_rows<R, R><<<tg, kBlock, 0, h->stream>>>(static_cast<const cx<R>*>(Y), ldy, Yr, n, kk);
  block_to_rows<R, R><<<tg, kBlock, 0, h->stream>>>(static_cast<const cx<R>*>(X), ldx, Xr, n, kk);
  h->launches += 2;
  if ((rc = bicgstab_core<R>(run, Yr, Xr, tol, maxit, false, nullptr)) != CCG_OK) return rc;
  zero_cols<R><<<256, kBlock, 0, h->stream>>>(Xr, n, kk, run.w.cols.zero_rhs);
  rows_to_block<R, R><<<tg, kBlock, 0, h->stream>>>(Xr, static_cast<cx<R>*>(X), ldx, n, kk);
  h->launches += 2;
  std::vector<int> st(kk);
  B_CUDA(cudaMemcpyAsync(st.data(), run.w.cols.status, kk * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  copy_cols_out(run.w.cols, kk, iters, status, relres, h->stream);
  B_CUDA(cudaStreamSynchronize(h->stream));
  timing_collect(h);
  if ((rc = tc_check_error(h)) != CCG_OK) return rc;
  if ((rc = oz_check_error(h)) != CCG_OK) return rc;
  return worst_status(st);
}

int solve_batched(ccg_handle* h, const ccg_operator* op, int64_t k, const void* Y, int64_t ldy, void* X, int64_t ldx,
                  double tol, int maxit, int32_t* iters, int32_t* status, double* relres) {
  if (op->dtype == CCG_C128) return batched_t<double>(h, op, k, Y, ldy, X, ldx, tol, maxit, iters, status, relres);
  return batched_t<float>(h, op, k, Y, ldy, X, ldx, tol, maxit, iters, status, relres);
}

// Y = A X for column-major device blocks (the multi-right-hand-side
// operator application on its own).
template <class R>
static int block_matvec_t(ccg_handle* h, const ccg_operator* op, int64_t k, const void* X, int64_t ldx, void* Y,
                          int64_t ldy) {
  const int64_t n = op->n;
  const int kk = (int)k;
  BRun<R> run;
  run.h = h; run.op = op; run.s = h->stream; run.n = n; run.k = kk; run.grid = phase_grid(h, n, kk);
  run.allow_tc = h->tc_mode >= 1;
  int rc = arena_reserve(h, BWs<R>::bytes(n, kk, 0, run.grid));
  if (rc != CCG_OK) return rc;
  run.w.carve(h->arena, n, kk, 0, run.grid);
  dim3 tg((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32));
  block_to_rows<R, R><<<tg, kBlock, 0, h->stream>>>(static_cast<const cx<R>*>(X), ldx, run.w.vec[6], n, kk);
  if ((rc = run.gemm(run.w.vec[6], run.w.vec[7], nullptr)) != CCG_OK) return rc;
  rows_to_block<R, R><<<tg, kBlock, 0, h->stream>>>(run.w.vec[7], static_cast<cx<R>*>(Y), ldy, n, kk);
  h->launches += 2;
  B_CUDA(cudaStreamSynchronize(h->stream));
  timing_collect(h);
  if ((rc = tc_check_error(h)) != CCG_OK) return rc;
  return oz_check_error(h);
}

int block_matvec(ccg_handle* h, const ccg_operator* op, int64_t k, const void* X, int64_t ldx, void* Y, int64_t ldy) {
  if (op->dtype == CCG_C128) return block_matvec_t<double>(h, op, k, X, ldx, Y, ldy);
  return block_matvec_t<float>(h, op, k, X, ldx, Y, ldy);
}

// X == 0 check: sets ctl->skip_mv when every entry of X is zero.
__global__ void all_zero(const double2* __restrict__ X, int64_t count, BCtl* ctl) {
  __shared__ int nz;
  if (threadIdx.x == 0) nz = 0;
  __syncthreads();
  int mine = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = X[e];
    mine |= (v.x != 0.0 || v.y != 0.0);
  }
  if (mine) atomicOr(&nz, 1);
  __syncthreads();
  if (threadIdx.x == 0 && nz) atomicExch(&ctl->skip_mv, 0);
}

int solve_batched_refined(ccg_handle* h, const ccg_operator* op, const ccg_operator* op_in, int64_t k, const void* Y,
                          int64_t ldy, void* X, int64_t ldx, double tol, int max_outer, double inner_tol,
                          int inner_maxit, int32_t* outer_out, int32_t* inner_out, int32_t* status, double* relres) {
  const int64_t n = op->n;
  const int kk = (int)k;
  cudaStream_t s = h->stream;
  BRun<double> ro;
  ro.h = h; ro.op = op; ro.s = s; ro.n = n; ro.k = kk; ro.grid = phase_grid(h, n, kk);
  BRun<float> ri;
  ri.h = h; ri.op = op_in; ri.s = s; ri.n = n; ri.k = kk; ri.grid = ro.grid;
  ri.allow_tc = h->tc_mode >= 1;
  const size_t b64 = al256(BWs<double>::bytes(n, kk, max_outer, ro.grid));
  int rc = arena_reserve(h, b64 + BWs<float>::bytes(n, kk, inner_maxit, ri.grid));
  if (rc != CCG_OK) return rc;
  ro.w.carve(h->arena, n, kk, max_outer, ro.grid);
  ri.w.carve(h->arena + b64, n, kk, inner_maxit, ri.grid);
  ro.red.partials = ro.w.partials; ro.red.counter = ro.w.counter;
  ri.red.partials = ri.w.partials; ri.red.counter = ri.w.counter;
  double2* Yr = ro.w.vec[0];
  double2* Xr = ro.w.vec[1];
  double2* AX = ro.w.vec[2];
  float2* R32 = ri.w.vec[6];
  float2* D32 = ri.w.vec[7];
  // complex64 blocks of the nested correction, in unused complex128 slots
  float2* E32 = reinterpret_cast<float2*>(ro.w.vec[3]);
  float2* AD32 = reinterpret_cast<float2*>(ro.w.vec[4]);
  float2* Rm = reinterpret_cast<float2*>(ro.w.vec[5]);
  dim3 tg((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32));
  block_to_rows<double, double><<<tg, kBlock, 0, s>>>(static_cast<const double2*>(Y), ldy, Yr, n, kk);
  block_to_rows<double, double><<<tg, kBlock, 0, s>>>(static_cast<const double2*>(X), ldx, Xr, n, kk);
  h->launches += 2;
  BCtl init;
  std::memset(&init, 0, sizeof(init));
  init.maxit = max_outer;
  init.tol = tol;
  init.skip_mv = 1;
  B_CUDA(cudaMemcpyAsync(ro.w.ctl, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  B_CUDA(cudaMemsetAsync(ro.w.counter, 0, ro.w.counter_bytes, s));
  B_CUDA(cudaMemsetAsync(ro.w.cols.done, 0, kk * sizeof(int), s));
  B_CUDA(cudaMemsetAsync(ro.w.cols.zero_rhs, 0, kk * sizeof(int), s));
  B_CUDA(cudaMemsetAsync(ro.w.cols.status, 0, kk * sizeof(int), s));
  B_CUDA(cudaMemsetAsync(ro.w.cols.bd, 0, kk * sizeof(int), s));
  // the first residual needs no product when X0 = 0
  all_zero<<<std::min<int64_t>((n * k + kBlock - 1) / kBlock, 1024), kBlock, 0, s>>>(Xr, n * k, ro.w.ctl);
  ++h->launches;
  std::vector<int> inner_it(kk, 0), inner_total(kk, 0);
  int outer = 0;
  B_CUDA(cudaMemcpyAsync(&init, ro.w.ctl, sizeof(init), cudaMemcpyDeviceToHost, s));
  B_CUDA(cudaStreamSynchronize(s));
  const bool x0_zero = init.skip_mv != 0;
  for (;; ++outer) {
    BRefResid p;
    p.n = n; p.k = kk; p.y = Yr; p.ax = AX; p.r32 = R32; p.d32 = D32; p.outer = outer;
    if (outer == 0 && x0_zero) p.ax = nullptr;   // R = Y: no product needed
    else if ((rc = ro.gemm(Xr, AX, nullptr)) != CCG_OK) return rc;
    ro.phase(p);
    B_CUDA(cudaGetLastError());
    int all = 0;
    B_CUDA(cudaMemcpyAsync(&all, &ro.w.ctl->all_done, sizeof(int), cudaMemcpyDeviceToHost, s));
    B_CUDA(cudaStreamSynchronize(s));
    if (all) break;
    // Correction D32 for A D = R32.  Split-bf16 tensor-core products are
    // ~1e-4 accurate at this size (their fp32 accumulation), so a
    // tensor-core solve is followed by one complex64 residual R32 - A D32
    // accurate to FP32 (the integer-slice tensor-core product, or CUDA
    // cores) and a second split-bf16 solve of it: the correction is then as
    // good as an inner solve with FP32-accurate products, with one such
    // product instead of one per iteration.
    const bool tc_inner = ri.allow_tc && tc_available(op_in);
    const int mid_steps = tc_inner ? 2 : 1;
    for (int mid = 0; mid < mid_steps; ++mid) {
      float2* rhs = mid == 0 ? R32 : Rm;
      float2* sol = mid == 0 ? D32 : E32;
      if ((rc = bicgstab_core<float>(ri, rhs, sol, inner_tol, inner_maxit, true, ro.w.cols.done)) != CCG_OK) return rc;
      B_CUDA(cudaMemcpyAsync(inner_it.data(), ri.w.cols.iters, kk * sizeof(int), cudaMemcpyDeviceToHost, s));
      B_CUDA(cudaStreamSynchronize(s));
      for (int c = 0; c < kk; ++c) inner_total[c] += inner_it[c];
      if (mid > 0) {
        BMidAdd a;
        a.n = n; a.k = kk; a.d = D32; a.e = E32;
        ro.phase(a);
      }
      if (mid + 1 < mid_steps) {
        ri.allow_tc = false;           // the FP32-accurate complex64 product
        if ((rc = ri.gemm(D32, AD32, nullptr)) != CCG_OK) return rc;
        ri.allow_tc = true;
        BMidResid m;
        m.n = n; m.k = kk; m.r = R32; m.ad = AD32; m.rm = Rm;
        ro.phase(m);
      }
    }
    BRefUpdate u;
    u.n = n; u.k = kk; u.x = Xr; u.d32 = D32;
    ro.phase(u);
  }
  zero_cols<double><<<256, kBlock, 0, s>>>(Xr, n, kk, ro.w.cols.zero_rhs);
  rows_to_block<double, double><<<tg, kBlock, 0, s>>>(Xr, static_cast<double2*>(X), ldx, n, kk);
  h->launches += 2;
  std::vector<int> st(kk);
  B_CUDA(cudaMemcpyAsync(st.data(), ro.w.cols.status, kk * sizeof(int), cudaMemcpyDeviceToHost, s));
  copy_cols_out(ro.w.cols, kk, outer_out, status, relres, s);
  B_CUDA(cudaStreamSynchronize(s));
  if (inner_out) std::memcpy(inner_out, inner_total.data(), kk * sizeof(int));
  timing_collect(h);
  if ((rc = tc_check_error(h)) != CCG_OK) return rc;
  if ((rc = oz_check_error(h)) != CCG_OK) return rc;
  return worst_status(st);
}

}  // namespace ccg
