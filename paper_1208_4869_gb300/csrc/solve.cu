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

namespace ccg {

// ---------------------------------------------------------------------------
// Phase kernel and accumulation helpers.
// ---------------------------------------------------------------------------
struct PhaseBase {
  static constexpr bool kReduce = true;
  __device__ __forceinline__ bool skip(const SolveState*) const { return false; }
  __device__ __forceinline__ void load(const SolveState*) {}
};

// One elementwise pass with its sums; A is the per-thread accumulator
// (double, or a float-float pair for complex64 data).
template <class P, class A>
__global__ void __launch_bounds__(kBlock) phase_kernel(P p, SolveState* st, Red red) {
  if (st->poll.done || p.skip(st)) return;
  p.load(st);
  A acc[P::NQ];
#pragma unroll
  for (int q = 0; q < P::NQ; ++q) acc_zero(acc[q]);
  const int64_t stride = (int64_t)gridDim.x * kBlock;
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < p.n; i += stride) p.element(i, acc);
  if (P::kReduce) {
    double tot[P::NQ];
    if (grid_reduce<P::NQ>(acc, red.partials, red.counter, tot) && threadIdx.x == 0) p.finish(tot, st);
  }
}

template <class T> __device__ __forceinline__ void acc_dotc(double* acc, T u, T v) {  // conj(u) v
  const double2 a = widen(u), b = widen(v);
  acc[0] += a.x * b.x + a.y * b.y;
  acc[1] += a.x * b.y - a.y * b.x;
}
template <class T> __device__ __forceinline__ void acc_dotu(double* acc, T u, T v) {  // u v
  const double2 a = widen(u), b = widen(v);
  acc[0] += a.x * b.x - a.y * b.y;
  acc[1] += a.x * b.y + a.y * b.x;
}
template <class T> __device__ __forceinline__ void acc_nrm2(double* acc, T u) {
  const double2 a = widen(u);
  acc[0] += a.x * a.x + a.y * a.y;
}
__device__ __forceinline__ void acc_dotc(FF* acc, float2 a, float2 b) {  // conj(a) b
  ff_add_prod(acc[0], a.x, b.x);
  ff_add_prod(acc[0], a.y, b.y);
  ff_add_prod(acc[1], a.x, b.y);
  ff_add_prod(acc[1], -a.y, b.x);
}
__device__ __forceinline__ void acc_dotu(FF* acc, float2 a, float2 b) {  // a b
  ff_add_prod(acc[0], a.x, b.x);
  ff_add_prod(acc[0], -a.y, b.y);
  ff_add_prod(acc[1], a.x, b.y);
  ff_add_prod(acc[1], a.y, b.x);
}
__device__ __forceinline__ void acc_nrm2(FF* acc, float2 a) {
  ff_add_prod(acc[0], a.x, a.x);
  ff_add_prod(acc[0], a.y, a.y);
}
template <class R> __device__ __forceinline__ bool tiny(double2 s) { return cabs(s) < tiny_guard<R>(); }
template <class R> __device__ __forceinline__ bool tiny(double s) { return fabs(s) < tiny_guard<R>(); }
__device__ __forceinline__ bool nonfinite(double v) { return !(v == v) || isinf(v); }

// Record the end of iteration k (residual rel).  The checks follow the
// methods' order: converged, then a breakdown found in this iteration
// (bd != 0), then the iteration cap.  Returns true if the solve stops.
__device__ __forceinline__ bool end_iteration(SolveState* st, int k, double rel, int bd) {
  st->poll.k = k;
  st->poll.relres = rel;
  st->hist[k] = rel;
  if (nonfinite(rel)) { st->poll.status = ST_NONFINITE; st->poll.done = 1; return true; }
  if (rel <= st->tol) { st->poll.status = ST_OK; st->poll.done = 1; return true; }
  if (bd) { st->poll.status = ST_BREAKDOWN; st->poll.breakdown = bd; st->poll.done = 1; return true; }
  if (k >= st->maxit) { st->poll.status = ST_NOT_CONVERGED; st->poll.done = 1; return true; }
  return false;
}
__device__ __forceinline__ void set_breakdown(SolveState* st, int which) {
  st->poll.status = ST_BREAKDOWN;
  st->poll.breakdown = which;
  st->poll.done = 1;
}

enum { M_BICGSTAB = CCG_BICGSTAB, M_CGNR = CCG_CGNR, M_QMR = CCG_QMR, M_COCG = CCG_COCG, M_COCR = CCG_COCR,
       M_BICG = CCG_BICG, M_GMRES = CCG_GMRES, M_CGS = CCG_CGS, M_CGNE = CCG_CGNE, M_TFQMR = CCG_TFQMR,
       M_BICGSTABL = CCG_BICGSTABL };

// Clears st->skip_mv (set to 1 beforehand) when any entry of x is nonzero.
template <class R> __global__ void __launch_bounds__(kBlock) x_zero_check(const cx<R>* __restrict__ x, int64_t n,
                                                                         SolveState* st) {
  int mine = 0;
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
    const cx<R> v = x[i];
    mine |= (v.x != (R)0 || v.y != (R)0);
  }
  if (__syncthreads_or(mine) && threadIdx.x == 0) st->skip_mv = 0;
}

// ---------------------------------------------------------------------------
// Start of every method: r = y - A x0, ||y||, ||r||, and the method's first
// scalars; the copies of r each method keeps (shadow vector, p, ...).
// ---------------------------------------------------------------------------
template <class R> struct InitR : PhaseBase {
  static constexpr int NQ = 5;  // ||y||^2, ||r||^2, non-finite count in y, [r, r]
  int64_t n;
  const cx<R>* y;
  MvOut<R> ax;
  cx<R>* r;
  cx<R>* c1;
  cx<R>* c2;
  int method;
  bool ax_zero;
  __device__ __forceinline__ void load(const SolveState* st) { ax_zero = st->skip_mv != 0; }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> yi = y[i];
    const cx<R> ri = ax_zero ? yi : csub(yi, ax.get(i));
    r[i] = ri;
    if (c1) c1[i] = ri;
    if (c2) c2[i] = ri;
    acc_nrm2(acc, yi);
    acc_nrm2(acc + 1, ri);
    if (!(isfinite((double)yi.x) && isfinite((double)yi.y))) acc_add1(acc[2]);
    if (method == M_COCG) acc_dotu(acc + 3, ri, ri);
  }
  __device__ void finish(const double* t, SolveState* st) {
    st->poll.k = 0;
    st->skip_mv = 0;
    if (t[2] != 0.0) { st->poll.status = ST_NONFINITE; st->poll.done = 1; return; }
    const double yn = sqrt(t[0]);
    st->poll.ynorm = yn;
    if (yn == 0.0) {
      st->zero_rhs = 1;
      st->hist[0] = 0.0;
      st->poll.relres = 0.0;
      st->poll.status = ST_OK;
      st->poll.done = 1;
      return;
    }
    const double rel = sqrt(t[1]) / yn;
    st->hist[0] = rel;
    st->poll.relres = rel;
    if (nonfinite(rel)) { st->poll.status = ST_NONFINITE; st->poll.done = 1; return; }
    if (rel <= st->tol) { st->poll.status = ST_OK; st->poll.done = 1; return; }
    if (st->maxit <= 0) { st->poll.status = ST_NOT_CONVERGED; st->poll.done = 1; return; }
    switch (method) {
      case M_BICGSTAB:
        st->rho = mkc(t[1], 0.0);  // <r^, r> with r^ = r
        st->rho_old = st->alpha = st->omega = mkc(1.0, 0.0);
        if (tiny<R>(st->rho)) set_breakdown(st, CCG_BD_RHO);
        break;
      case M_QMR:
        st->qrho = st->xi = sqrt(t[1]);  // ||v~_1|| = ||w~_1|| = ||r_0||
        st->gamma_prev = 1.0;
        st->theta_prev = 0.0;
        st->eta = mkc(-1.0, 0.0);
        st->eps = mkc(0.0, 0.0);
        if (tiny<R>(st->qrho)) set_breakdown(st, CCG_BD_RHO);
        break;
      case M_COCG:
        st->rho = mkc(t[3], t[4]);
        if (tiny<R>(st->rho)) set_breakdown(st, CCG_BD_RHO);
        break;
      case M_BICG:
        st->rho = mkc(t[1], 0.0);  // <r~, r> with r~ = r
        if (tiny<R>(st->rho)) set_breakdown(st, CCG_BD_RHO);
        break;
      case M_GMRES:
        st->gm_beta = sqrt(t[1]);
        break;
      case M_CGS:
        st->rho = mkc(t[1], 0.0);  // <r^, r> with r^ = r
        if (tiny<R>(st->rho)) set_breakdown(st, CCG_BD_RHO);
        break;
      case M_CGNE:
        st->gamma = t[1];          // ||r||^2
        break;
      case M_BICGSTABL:
        st->rho_old = mkc(1.0, 0.0);  // rho_0
        st->alpha = mkc(0.0, 0.0);
        st->omega = mkc(1.0, 0.0);
        break;
      case M_TFQMR:
        st->tau = sqrt(t[1]);
        st->theta = 0.0;
        st->eta = mkc(0.0, 0.0);
        st->rho = mkc(t[1], 0.0);  // <r^, r_0> with r^ = r_0
        break;
      default:  // COCR forms its first scalars after the product A r0
        break;
    }
  }
};

// ||y - A x||^2 for the final true residual.
template <class R> struct TrueRes : PhaseBase {
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* y;
  MvOut<R> ax;
  double* out;
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) { acc_nrm2(acc, csub(y[i], ax.get(i))); }
  __device__ void finish(const double* t, SolveState*) { *out = t[0]; }
};

// Standalone pieces of the C ABI: sum of partials, and a dot product.
template <class R> struct SumParts : PhaseBase {
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  MvOut<R> mv;
  cx<R>* y;
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) { y[i] = mv.get(i); }
  __device__ void finish(const double*, SolveState*) {}
};
template <class R> struct DotPhase : PhaseBase {
  static constexpr int NQ = 2;
  int64_t n;
  const cx<R>* u;
  const cx<R>* v;
  int conj;
  double* out;
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    if (conj) acc_dotc(acc, u[i], v[i]);
    else acc_dotu(acc, u[i], v[i]);
  }
  __device__ void finish(const double* t, SolveState*) { out[0] = t[0]; out[1] = t[1]; }
};

// ---------------------------------------------------------------------------
// BiCGSTAB (van der Vorst; PIM `bicgstab`).
// ---------------------------------------------------------------------------
template <class R> struct BiP : PhaseBase {  // p = r, or p = r + beta (p - omega v)
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* r;
  cx<R>* p;
  const cx<R>* v;
  cx<R> beta, omega;
  bool first;
  __device__ __forceinline__ void load(const SolveState* st) {
    first = st->poll.k == 0;
    beta = narrow<R>(st->beta);
    omega = narrow<R>(st->omega);
  }
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) {
    p[i] = first ? r[i] : cadd(r[i], cmul(beta, csub(p[i], cmul(omega, v[i]))));
  }
  __device__ void finish(const double*, SolveState*) {}
};
template <class R> struct BiSigma : PhaseBase {  // sigma = <r^, v>, alpha = rho / sigma
  static constexpr int NQ = 2;
  int64_t n;
  MvOut<R> mv;
  cx<R>* v;
  const cx<R>* rh;
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> vi = mv.get(i);
    if (mv.P) v[i] = vi;
    acc_dotc(acc, rh[i], vi);
  }
  __device__ void finish(const double* t, SolveState* st) {
    const double2 sigma = mkc(t[0], t[1]);
    if (tiny<R>(sigma)) { set_breakdown(st, CCG_BD_SIGMA); return; }
    st->alpha = cdiv(st->rho, sigma);
  }
};
template <class R> struct BiS : PhaseBase {  // s = r - alpha v; half-step exit when ||s|| meets tol
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* r;
  const cx<R>* v;
  cx<R>* s;
  cx<R> alpha;
  __device__ __forceinline__ void load(const SolveState* st) { alpha = narrow<R>(st->alpha); }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> si = csub(r[i], cmul(alpha, v[i]));
    s[i] = si;
    acc_nrm2(acc, si);
  }
  __device__ void finish(const double* t, SolveState* st) {
    st->snorm = sqrt(t[0]) / st->poll.ynorm;
    st->half = st->snorm <= st->tol ? 1 : 0;
  }
};
template <class R> struct BiOmega : PhaseBase {  // omega = <t, s> / <t, t>
  static constexpr int NQ = 3;
  int64_t n;
  MvOut<R> mv;
  cx<R>* t;
  const cx<R>* s;
  __device__ __forceinline__ bool skip(const SolveState* st) const { return st->half != 0; }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> ti = mv.get(i);
    if (mv.P) t[i] = ti;
    acc_dotc(acc, ti, s[i]);
    acc_nrm2(acc + 2, ti);
  }
  __device__ void finish(const double* q, SolveState* st) {
    const double tt = q[2];
    if (tiny<R>(tt)) { set_breakdown(st, CCG_BD_TT); return; }
    st->omega = mkc(q[0] / tt, q[1] / tt);
  }
};
template <class R> struct BiXR : PhaseBase {  // x += alpha p + omega s; r = s - omega t; next rho = <r^, r>
  static constexpr int NQ = 3;
  int64_t n;
  cx<R>* x;
  cx<R>* r;
  const cx<R>* p;
  const cx<R>* s;
  const cx<R>* t;
  const cx<R>* rh;
  cx<R> alpha, omega;
  bool half;
  __device__ __forceinline__ void load(const SolveState* st) {
    half = st->half != 0;
    alpha = narrow<R>(st->alpha);
    omega = narrow<R>(st->omega);
  }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    if (half) {
      x[i] = cadd(x[i], cmul(alpha, p[i]));
      return;
    }
    x[i] = cadd(x[i], cadd(cmul(alpha, p[i]), cmul(omega, s[i])));
    const cx<R> ri = csub(s[i], cmul(omega, t[i]));
    r[i] = ri;
    acc_dotc(acc, rh[i], ri);
    acc_nrm2(acc + 2, ri);
  }
  __device__ void finish(const double* q, SolveState* st) {
    const int k = st->poll.k + 1;
    if (st->half) {
      st->poll.k = k;
      st->poll.relres = st->snorm;
      st->hist[k] = st->snorm;
      st->poll.status = ST_OK;
      st->poll.done = 1;
      return;
    }
    const double rel = sqrt(q[2]) / st->poll.ynorm;
    if (end_iteration(st, k, rel, tiny<R>(st->omega) ? CCG_BD_OMEGA : 0)) return;
    const double2 rho_new = mkc(q[0], q[1]);
    if (tiny<R>(rho_new)) { set_breakdown(st, CCG_BD_RHO); return; }
    st->beta = cmul(cdiv(rho_new, st->rho), cdiv(st->alpha, st->omega));
    st->rho_old = st->rho;
    st->rho = rho_new;
  }
};

// ---------------------------------------------------------------------------
// CGNR (PIM `cgnr`): CG on A^H A x = A^H y, residual r = y - A x.
// ---------------------------------------------------------------------------
template <class R> struct CgZ : PhaseBase {  // z = A^H r (from partials), gamma' = ||z||^2; first: p = z
  static constexpr int NQ = 1;
  int64_t n;
  MvOut<R> mv;
  cx<R>* z;
  cx<R>* p;  // non-null on the first call
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> zi = mv.get(i);
    if (mv.P) z[i] = zi;
    if (p) p[i] = zi;
    acc_nrm2(acc, zi);
  }
  __device__ void finish(const double* t, SolveState* st) {
    const double g = t[0];
    if (st->poll.k > 0) st->beta = mkc(g / st->gamma, 0.0);
    st->gamma = g;
    if (tiny<R>(g)) set_breakdown(st, CCG_BD_GAMMA);
  }
};
template <class R> struct CgAlpha : PhaseBase {  // w = A p, alpha = gamma / ||w||^2
  static constexpr int NQ = 1;
  int64_t n;
  MvOut<R> mv;
  cx<R>* w;
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> wi = mv.get(i);
    if (mv.P) w[i] = wi;
    acc_nrm2(acc, wi);
  }
  __device__ void finish(const double* t, SolveState* st) {
    if (tiny<R>(t[0])) { set_breakdown(st, CCG_BD_WW); return; }
    st->alpha = mkc(st->gamma / t[0], 0.0);
  }
};
template <class R> struct CgXR : PhaseBase {  // x += alpha p; r -= alpha w
  static constexpr int NQ = 1;
  int64_t n;
  cx<R>* x;
  cx<R>* r;
  const cx<R>* p;
  const cx<R>* w;
  R alpha;
  __device__ __forceinline__ void load(const SolveState* st) { alpha = (R)st->alpha.x; }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    x[i] = cadd(x[i], cscale(alpha, p[i]));
    const cx<R> ri = csub(r[i], cscale(alpha, w[i]));
    r[i] = ri;
    acc_nrm2(acc, ri);
  }
  __device__ void finish(const double* t, SolveState* st) {
    end_iteration(st, st->poll.k + 1, sqrt(t[0]) / st->poll.ynorm, 0);
  }
};
template <class R> struct CgP : PhaseBase {  // p = z + beta p
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* z;
  cx<R>* p;
  R beta;
  __device__ __forceinline__ void load(const SolveState* st) { beta = (R)st->beta.x; }
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) { p[i] = cadd(z[i], cscale(beta, p[i])); }
  __device__ void finish(const double*, SolveState*) {}
};

// ---------------------------------------------------------------------------
// QMR without look-ahead, coupled two-term recurrences (Freund-Nachtigal;
// PIM `qmr`), complex form with A^H.
// ---------------------------------------------------------------------------
template <class R> __device__ __forceinline__ void qmr_pq_coefs(SolveState* st) {
  // cp = xi delta / eps, cq = conj(rho delta / eps), for iterations after the first
  st->cp = cdiv(cscale(st->xi, st->delta), st->eps);
  st->cq = cconj(cdiv(cscale(st->qrho, st->delta), st->eps));
}
template <class R> struct QVW : PhaseBase {  // first iteration: v = v~/rho, w = w~/xi, delta = <w, v>
  static constexpr int NQ = 2;
  int64_t n;
  const cx<R>* vt;
  const cx<R>* wt;
  cx<R>* v;
  cx<R>* w;
  R rinv, xinv;
  __device__ __forceinline__ void load(const SolveState* st) {
    rinv = (R)(1.0 / st->qrho);
    xinv = (R)(1.0 / st->xi);
  }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> vi = cscale(rinv, vt[i]), wi = cscale(xinv, wt[i]);
    v[i] = vi;
    w[i] = wi;
    acc_dotc(acc, wi, vi);
  }
  __device__ void finish(const double* t, SolveState* st) {
    st->delta = mkc(t[0], t[1]);
    if (tiny<R>(st->delta)) set_breakdown(st, CCG_BD_DELTA);
  }
};
template <class R> struct QPQ : PhaseBase {  // p = v - cp p, q = w - cq q (first: p = v, q = w)
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* v;
  const cx<R>* w;
  cx<R>* p;
  cx<R>* q;
  cx<R> cp, cq;
  bool first;
  __device__ __forceinline__ void load(const SolveState* st) {
    first = st->poll.k == 0;
    cp = narrow<R>(st->cp);
    cq = narrow<R>(st->cq);
  }
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) {
    if (first) {
      p[i] = v[i];
      q[i] = w[i];
    } else {
      p[i] = csub(v[i], cmul(cp, p[i]));
      q[i] = csub(w[i], cmul(cq, q[i]));
    }
  }
  __device__ void finish(const double*, SolveState*) {}
};
template <class R> struct QEps : PhaseBase {  // p~ = A p, u = A^H q; eps = <q, p~>, beta = eps / delta
  static constexpr int NQ = 2;
  int64_t n;
  MvOut<R> mv1, mv2;
  cx<R>* pt;
  cx<R>* u;
  const cx<R>* q;
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> pti = mv1.get(i), ui = mv2.get(i);
    if (mv1.P) pt[i] = pti;
    if (mv2.P) u[i] = ui;
    acc_dotc(acc, q[i], pti);
  }
  __device__ void finish(const double* t, SolveState* st) {
    const double2 eps = mkc(t[0], t[1]);
    if (tiny<R>(eps)) { set_breakdown(st, CCG_BD_EPS); return; }
    st->eps = eps;
    st->beta = cdiv(eps, st->delta);
    if (tiny<R>(st->beta)) set_breakdown(st, CCG_BD_BETA);
  }
};
template <class R> struct QVT : PhaseBase {  // v~ = p~ - beta v, w~ = u - conj(beta) w; theta, gamma, eta
  static constexpr int NQ = 2;
  int64_t n;
  const cx<R>* pt;
  const cx<R>* u;
  const cx<R>* v;
  const cx<R>* w;
  cx<R>* vt;
  cx<R>* wt;
  cx<R> beta, betac;
  __device__ __forceinline__ void load(const SolveState* st) {
    beta = narrow<R>(st->beta);
    betac = cconj(beta);
  }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> a = csub(pt[i], cmul(beta, v[i])), b = csub(u[i], cmul(betac, w[i]));
    vt[i] = a;
    wt[i] = b;
    acc_nrm2(acc, a);
    acc_nrm2(acc + 1, b);
  }
  __device__ void finish(const double* t, SolveState* st) {
    st->rho_n = sqrt(t[0]);
    st->xi_n = sqrt(t[1]);
    const double theta = st->rho_n / (st->gamma_prev * cabs(st->beta));
    const double gamma = 1.0 / sqrt(1.0 + theta * theta);
    if (tiny<R>(gamma)) { set_breakdown(st, CCG_BD_GAMMA); return; }
    // eta = -eta rho gamma^2 / (beta gamma_prev^2)
    const double2 num = cscale(st->qrho * gamma * gamma, mkc(-st->eta.x, -st->eta.y));
    st->eta = cdiv(num, cscale(st->gamma_prev * st->gamma_prev, st->beta));
    st->c = (st->theta_prev * gamma) * (st->theta_prev * gamma);
    st->theta = theta;
    st->gamma = gamma;
  }
};
template <class R> struct QDX : PhaseBase {
  // d = eta p + c d, s = eta p~ + c s (first: d = eta p, s = eta p~); x += d; r -= s;
  // and the start of the next iteration: v = v~/rho', w = w~/xi', delta' = <w, v>.
  static constexpr int NQ = 3;
  int64_t n;
  const cx<R>* p;
  const cx<R>* pt;
  cx<R>* d;
  cx<R>* s;
  cx<R>* x;
  cx<R>* r;
  const cx<R>* vt;
  const cx<R>* wt;
  cx<R>* v;
  cx<R>* w;
  cx<R> eta;
  R c, rinv, xinv;
  bool first;
  __device__ __forceinline__ void load(const SolveState* st) {
    first = st->poll.k == 0;
    eta = narrow<R>(st->eta);
    c = (R)st->c;
    rinv = (R)(1.0 / st->rho_n);
    xinv = (R)(1.0 / st->xi_n);
  }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    cx<R> di = cmul(eta, p[i]), si = cmul(eta, pt[i]);
    if (!first) {
      di = cadd(di, cscale(c, d[i]));
      si = cadd(si, cscale(c, s[i]));
    }
    d[i] = di;
    s[i] = si;
    x[i] = cadd(x[i], di);
    const cx<R> ri = csub(r[i], si);
    r[i] = ri;
    acc_nrm2(acc, ri);
    const cx<R> vi = cscale(rinv, vt[i]), wi = cscale(xinv, wt[i]);
    v[i] = vi;
    w[i] = wi;
    acc_dotc(acc + 1, wi, vi);
  }
  __device__ void finish(const double* t, SolveState* st) {
    if (end_iteration(st, st->poll.k + 1, sqrt(t[0]) / st->poll.ynorm, 0)) return;
    st->qrho = st->rho_n;
    st->xi = st->xi_n;
    st->gamma_prev = st->gamma;
    st->theta_prev = st->theta;
    if (tiny<R>(st->qrho)) { set_breakdown(st, CCG_BD_RHO); return; }
    if (tiny<R>(st->xi)) { set_breakdown(st, CCG_BD_XI); return; }
    st->delta = mkc(t[1], t[2]);
    if (tiny<R>(st->delta)) { set_breakdown(st, CCG_BD_DELTA); return; }
    qmr_pq_coefs<R>(st);
  }
};
// ---------------------------------------------------------------------------
// COCG: complex-symmetric CG with [u, v] = sum u_i v_i (Sec. 2.2 reading).
// ---------------------------------------------------------------------------
template <class R> struct CoMu : PhaseBase {  // q = A p, mu = [p, q], alpha = rho / mu
  static constexpr int NQ = 2;
  int64_t n;
  MvOut<R> mv;
  cx<R>* q;
  const cx<R>* p;
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> qi = mv.get(i);
    if (mv.P) q[i] = qi;
    acc_dotu(acc, p[i], qi);
  }
  __device__ void finish(const double* t, SolveState* st) {
    const double2 mu = mkc(t[0], t[1]);
    if (tiny<R>(mu)) { set_breakdown(st, CCG_BD_MU); return; }
    st->alpha = cdiv(st->rho, mu);
  }
};
template <class R> struct CoXR : PhaseBase {  // x += alpha p; r -= alpha q; rho' = [r, r], beta = rho'/rho
  static constexpr int NQ = 3;
  int64_t n;
  cx<R>* x;
  cx<R>* r;
  const cx<R>* p;
  const cx<R>* q;
  cx<R> alpha;
  __device__ __forceinline__ void load(const SolveState* st) { alpha = narrow<R>(st->alpha); }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    x[i] = cadd(x[i], cmul(alpha, p[i]));
    const cx<R> ri = csub(r[i], cmul(alpha, q[i]));
    r[i] = ri;
    acc_nrm2(acc, ri);
    acc_dotu(acc + 1, ri, ri);
  }
  __device__ void finish(const double* t, SolveState* st) {
    if (end_iteration(st, st->poll.k + 1, sqrt(t[0]) / st->poll.ynorm, 0)) return;
    const double2 rho_new = mkc(t[1], t[2]);
    if (tiny<R>(rho_new)) { set_breakdown(st, CCG_BD_RHO); return; }
    st->beta = cdiv(rho_new, st->rho);
    st->rho = rho_new;
  }
};
template <class R> struct CoP : PhaseBase {  // p = r + beta p
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* r;
  cx<R>* p;
  cx<R> beta;
  __device__ __forceinline__ void load(const SolveState* st) { beta = narrow<R>(st->beta); }
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) { p[i] = cadd(r[i], cmul(beta, p[i])); }
  __device__ void finish(const double*, SolveState*) {}
};

// ---------------------------------------------------------------------------
// COCR (Sogabe-Zhang; Sec. 3.4): one product w = A r per iteration, q = A p
// carried by recurrence, unconjugated form.
// ---------------------------------------------------------------------------
template <class R> struct CrRho : PhaseBase {  // w = A r; rho' = [r, w]; beta = rho' / rho after the first
  static constexpr int NQ = 2;
  int64_t n;
  MvOut<R> mv;
  cx<R>* w;
  const cx<R>* r;
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> wi = mv.get(i);
    if (mv.P) w[i] = wi;
    acc_dotu(acc, r[i], wi);
  }
  __device__ void finish(const double* t, SolveState* st) {
    const double2 rho_new = mkc(t[0], t[1]);
    if (tiny<R>(rho_new)) { set_breakdown(st, CCG_BD_RHO); return; }
    if (st->poll.k > 0) st->beta = cdiv(rho_new, st->rho);
    st->rho = rho_new;
  }
};
template <class R> struct CrPQ : PhaseBase {  // p = r + beta p, q = w + beta q (first: p = r, q = w); mu = [q, q]
  static constexpr int NQ = 2;
  int64_t n;
  const cx<R>* r;
  const cx<R>* w;
  cx<R>* p;
  cx<R>* q;
  cx<R> beta;
  bool first;
  __device__ __forceinline__ void load(const SolveState* st) {
    first = st->poll.k == 0;
    beta = narrow<R>(st->beta);
  }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    cx<R> pi = r[i], qi = w[i];
    if (!first) {
      pi = cfma(beta, p[i], pi);
      qi = cfma(beta, q[i], qi);
    }
    p[i] = pi;
    q[i] = qi;
    acc_dotu(acc, qi, qi);
  }
  __device__ void finish(const double* t, SolveState* st) {
    const double2 mu = mkc(t[0], t[1]);
    if (tiny<R>(mu)) { set_breakdown(st, CCG_BD_MU); return; }
    st->alpha = cdiv(st->rho, mu);
  }
};
template <class R> struct CrXR : PhaseBase {  // x += alpha p; r -= alpha q
  static constexpr int NQ = 1;
  int64_t n;
  cx<R>* x;
  cx<R>* r;
  const cx<R>* p;
  const cx<R>* q;
  cx<R> alpha;
  __device__ __forceinline__ void load(const SolveState* st) { alpha = narrow<R>(st->alpha); }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    x[i] = cadd(x[i], cmul(alpha, p[i]));
    const cx<R> ri = csub(r[i], cmul(alpha, q[i]));
    r[i] = ri;
    acc_nrm2(acc, ri);
  }
  __device__ void finish(const double* t, SolveState* st) {
    end_iteration(st, st->poll.k + 1, sqrt(t[0]) / st->poll.ynorm, 0);
  }
};

// ---------------------------------------------------------------------------
// BiCG (Fletcher; PIM `bigcg`, Sec. 2.1): A p and A^H p~ from one read of a
// dense A, conjugated products, shadow r~_0 = r_0.
// ---------------------------------------------------------------------------
template <class R> struct BgP : PhaseBase {  // p = r + beta p, p~ = r~ + conj(beta) p~ (first: p = r, p~ = r~)
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* r;
  const cx<R>* rt;
  cx<R>* p;
  cx<R>* pt;
  cx<R> beta;
  bool first;
  __device__ __forceinline__ void load(const SolveState* st) {
    first = st->poll.k == 0;
    beta = narrow<R>(st->beta);
  }
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) {
    if (first) {
      p[i] = r[i];
      pt[i] = rt[i];
    } else {
      p[i] = cfma(beta, p[i], r[i]);
      pt[i] = cfma(cconj(beta), pt[i], rt[i]);
    }
  }
  __device__ void finish(const double*, SolveState*) {}
};
template <class R> struct BgSigma : PhaseBase {  // q = A p, q~ = A^H p~; sigma = <p~, q>, alpha = rho / sigma
  static constexpr int NQ = 2;
  int64_t n;
  MvOut<R> mv1, mv2;
  cx<R>* q;
  cx<R>* qt;
  const cx<R>* pt;
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> qi = mv1.get(i), qti = mv2.get(i);
    if (mv1.P) q[i] = qi;
    if (mv2.P) qt[i] = qti;
    acc_dotc(acc, pt[i], qi);
  }
  __device__ void finish(const double* t, SolveState* st) {
    const double2 sigma = mkc(t[0], t[1]);
    if (tiny<R>(sigma)) { set_breakdown(st, CCG_BD_SIGMA); return; }
    st->alpha = cdiv(st->rho, sigma);
  }
};
template <class R> struct BgXR : PhaseBase {  // x += alpha p; r -= alpha q; r~ -= conj(alpha) q~; rho' = <r~, r>
  static constexpr int NQ = 3;
  int64_t n;
  cx<R>* x;
  cx<R>* r;
  cx<R>* rt;
  const cx<R>* p;
  const cx<R>* q;
  const cx<R>* qt;
  cx<R> alpha;
  __device__ __forceinline__ void load(const SolveState* st) { alpha = narrow<R>(st->alpha); }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    x[i] = cadd(x[i], cmul(alpha, p[i]));
    const cx<R> ri = csub(r[i], cmul(alpha, q[i]));
    const cx<R> rti = csub(rt[i], cmul(cconj(alpha), qt[i]));
    r[i] = ri;
    rt[i] = rti;
    acc_nrm2(acc, ri);
    acc_dotc(acc + 1, rti, ri);
  }
  __device__ void finish(const double* t, SolveState* st) {
    if (end_iteration(st, st->poll.k + 1, sqrt(t[0]) / st->poll.ynorm, 0)) return;
    const double2 rho_new = mkc(t[1], t[2]);
    if (tiny<R>(rho_new)) { set_breakdown(st, CCG_BD_RHO); return; }
    st->beta = cdiv(rho_new, st->rho);
    st->rho = rho_new;
  }
};

// ---------------------------------------------------------------------------
// CGS (Sonneveld; PIM `cgs`, Sec. 2.1): two products per iteration,
// conjugated products, shadow r^ = r_0.
// ---------------------------------------------------------------------------
template <class R> struct CsUP : PhaseBase {  // u = r + beta q, p = u + beta (q + beta p) (first: u = p = r)
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* r;
  const cx<R>* q;
  cx<R>* u;
  cx<R>* p;
  cx<R> beta;
  bool first;
  __device__ __forceinline__ void load(const SolveState* st) {
    first = st->poll.k == 0;
    beta = narrow<R>(st->beta);
  }
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) {
    if (first) {
      u[i] = r[i];
      p[i] = r[i];
    } else {
      const cx<R> qi = q[i];
      const cx<R> ui = cfma(beta, qi, r[i]);
      u[i] = ui;
      p[i] = cfma(beta, cfma(beta, p[i], qi), ui);
    }
  }
  __device__ void finish(const double*, SolveState*) {}
};
template <class R> struct CsSigma : PhaseBase {  // v = A p; sigma = <r^, v>, alpha = rho / sigma
  static constexpr int NQ = 2;
  int64_t n;
  MvOut<R> mv;
  cx<R>* v;
  const cx<R>* rh;
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> vi = mv.get(i);
    if (mv.P) v[i] = vi;
    acc_dotc(acc, rh[i], vi);
  }
  __device__ void finish(const double* t, SolveState* st) {
    const double2 sigma = mkc(t[0], t[1]);
    if (tiny<R>(sigma)) { set_breakdown(st, CCG_BD_SIGMA); return; }
    st->alpha = cdiv(st->rho, sigma);
  }
};
template <class R> struct CsQ : PhaseBase {  // q = u - alpha v; u^ = u + q; x += alpha u^
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* u;
  const cx<R>* v;
  cx<R>* q;
  cx<R>* uh;
  cx<R>* x;
  cx<R> alpha;
  __device__ __forceinline__ void load(const SolveState* st) { alpha = narrow<R>(st->alpha); }
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) {
    const cx<R> ui = u[i];
    const cx<R> qi = csub(ui, cmul(alpha, v[i]));
    const cx<R> uhi = cadd(ui, qi);
    q[i] = qi;
    uh[i] = uhi;
    x[i] = cadd(x[i], cmul(alpha, uhi));
  }
  __device__ void finish(const double*, SolveState*) {}
};
template <class R> struct CsR : PhaseBase {  // r -= alpha A u^; rho' = <r^, r>, beta = rho' / rho
  static constexpr int NQ = 3;
  int64_t n;
  MvOut<R> mv;
  cx<R>* r;
  const cx<R>* rh;
  cx<R> alpha;
  __device__ __forceinline__ void load(const SolveState* st) { alpha = narrow<R>(st->alpha); }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> ri = csub(r[i], cmul(alpha, mv.get(i)));
    r[i] = ri;
    acc_nrm2(acc, ri);
    acc_dotc(acc + 1, rh[i], ri);
  }
  __device__ void finish(const double* t, SolveState* st) {
    if (end_iteration(st, st->poll.k + 1, sqrt(t[0]) / st->poll.ynorm, 0)) return;
    const double2 rho_new = mkc(t[1], t[2]);
    if (tiny<R>(rho_new)) { set_breakdown(st, CCG_BD_RHO); return; }
    st->beta = cdiv(rho_new, st->rho);
    st->rho = rho_new;
  }
};

// ---------------------------------------------------------------------------
// CGNE (Craig's method; PIM `cgne`, Sec. 2.1): CG on A A^H u = y carried in
// x = A^H u; products A p and A^H r per iteration.
// ---------------------------------------------------------------------------
template <class R> struct CnXR : PhaseBase {  // w = A p; x += alpha p; r -= alpha w; gamma' = ||r||^2
  static constexpr int NQ = 1;
  int64_t n;
  MvOut<R> mv;
  cx<R>* x;
  cx<R>* r;
  const cx<R>* p;
  R alpha;
  __device__ __forceinline__ void load(const SolveState* st) { alpha = (R)st->alpha.x; }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    x[i] = cadd(x[i], cscale(alpha, p[i]));
    const cx<R> ri = csub(r[i], cscale(alpha, mv.get(i)));
    r[i] = ri;
    acc_nrm2(acc, ri);
  }
  __device__ void finish(const double* t, SolveState* st) {
    if (end_iteration(st, st->poll.k + 1, sqrt(t[0]) / st->poll.ynorm, 0)) return;
    st->beta = mkc(t[0] / st->gamma, 0.0);
    st->gamma = t[0];
  }
};
template <class R> struct CnP : PhaseBase {  // z = A^H r; p = z + beta p (first: p = z); alpha = gamma / ||p||^2
  static constexpr int NQ = 1;
  int64_t n;
  MvOut<R> mv;
  cx<R>* p;
  R beta;
  bool first;
  __device__ __forceinline__ void load(const SolveState* st) {
    first = st->poll.k == 0;
    beta = (R)st->beta.x;
  }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> zi = mv.get(i);
    const cx<R> pi = first ? zi : cadd(zi, cscale(beta, p[i]));
    p[i] = pi;
    acc_nrm2(acc, pi);
  }
  __device__ void finish(const double* t, SolveState* st) {
    if (tiny<R>(t[0])) { set_breakdown(st, CCG_BD_WW); return; }
    st->alpha = mkc(st->gamma / t[0], 0.0);
  }
};

// ---------------------------------------------------------------------------
// TFQMR (Freund; PIM `tfqmr`, Sec. 2.1), two half-steps per iteration,
// conjugated products, shadow r^ = r_0.  The step x += eta d of a half-step
// needs eta, which its own reduction forms, so it is applied in the next
// half-step's pass; TqXStop applies it instead when the solve stops (or
// breaks down) first, and ends the solve.  `half` marks that pending stop.
// ---------------------------------------------------------------------------
// theta^2 eta / alpha, the weight of d in d = u_m + (theta^2 eta / alpha) d.
__device__ __forceinline__ double2 tq_f(const SolveState* st) {
  return cmul(cdiv(mkc(st->theta * st->theta, 0.0), st->alpha), st->eta);
}
// Quasi-residual update after ||w||^2 = ww in half-step m (0-based) of
// iteration k; records the bound sqrt(m + 2) tau / ||y||.  True if stopping.
__device__ __forceinline__ bool tq_update(SolveState* st, double ww, int m, int k, bool odd) {
  const double theta = sqrt(ww) / st->tau;
  const double c = 1.0 / sqrt(1.0 + theta * theta);
  st->tau = st->tau * theta * c;
  st->theta = theta;
  st->eta = cscale(c * c, st->alpha);
  const double rel = st->tau * sqrt(m + 2.0) / st->poll.ynorm;
  st->hist[k] = rel;
  st->poll.relres = rel;
  int status = -100;
  if (nonfinite(rel)) status = ST_NONFINITE;
  else if (rel <= st->tol) status = ST_OK;
  else if (odd && k >= st->maxit) status = ST_NOT_CONVERGED;
  if (odd || status != -100) st->poll.k = k;
  if (status == -100) return false;
  st->poll.status = status;
  st->half = 1;
  return true;
}
template <class R> struct TqInit : PhaseBase {  // v = 0, d = 0 (v gains A u in TqSigma)
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  cx<R>* v;
  cx<R>* d;
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) {
    v[i] = mk<R>(0, 0);
    d[i] = mk<R>(0, 0);
  }
  __device__ void finish(const double*, SolveState*) {}
};
template <class R> struct TqSigma : PhaseBase {  // v += A u; sigma = <r^, v>, alpha = rho / sigma
  static constexpr int NQ = 2;
  int64_t n;
  MvOut<R> mv;
  cx<R>* v;
  const cx<R>* rh;
  __device__ __forceinline__ bool skip(const SolveState* st) const { return st->half != 0; }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> vi = cadd(v[i], mv.get(i));
    v[i] = vi;
    acc_dotc(acc, rh[i], vi);
  }
  __device__ void finish(const double* t, SolveState* st) {
    const double2 sigma = mkc(t[0], t[1]);
    if (tiny<R>(sigma)) {  // the pending x step still applies
      st->poll.status = ST_BREAKDOWN;
      st->poll.breakdown = CCG_BD_SIGMA;
      st->half = 1;
      return;
    }
    st->alpha = cdiv(st->rho, sigma);
  }
};
// One half-step: x += eta d (the previous half-step's); even: u_{m+1} =
// u_m - alpha v; w -= alpha A u_m; d = u_m + f d; ||w||^2 (odd: also <r^, w>).
template <class R, bool ODD> struct TqHalf : PhaseBase {
  static constexpr int NQ = ODD ? 3 : 1;
  int64_t n;
  cx<R>* x;
  cx<R>* w;
  cx<R>* d;
  const cx<R>* um;   // u_m
  cx<R>* un;         // even: u_{m+1} = u_m - alpha v
  const cx<R>* v;
  const cx<R>* uh;   // A u_m
  const cx<R>* rh;
  cx<R> alpha, eta, f;
  __device__ __forceinline__ bool skip(const SolveState* st) const { return st->half != 0; }
  __device__ __forceinline__ void load(const SolveState* st) {
    alpha = narrow<R>(st->alpha);
    eta = narrow<R>(st->eta);
    f = narrow<R>(tq_f(st));
  }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> di = d[i], umi = um[i];
    x[i] = cadd(x[i], cmul(eta, di));
    if (!ODD) un[i] = csub(umi, cmul(alpha, v[i]));
    const cx<R> wi = csub(w[i], cmul(alpha, uh[i]));
    w[i] = wi;
    d[i] = cadd(umi, cmul(f, di));
    acc_nrm2(acc, wi);
    if (ODD) acc_dotc(acc + 1, rh[i], wi);
  }
  __device__ void finish(const double* t, SolveState* st) {
    const int k = st->poll.k + 1;
    if (tq_update(st, t[0], ODD ? 2 * k - 1 : 2 * k - 2, k, ODD) || !ODD) return;
    const double2 rho_new = mkc(t[1], t[2]);
    if (tiny<R>(rho_new)) {
      st->poll.status = ST_BREAKDOWN;
      st->poll.breakdown = CCG_BD_RHO;
      st->half = 1;
      return;
    }
    st->beta = cdiv(rho_new, st->rho);
    st->rho = rho_new;
  }
};
template <class R> struct TqXStop : PhaseBase {  // after a stop: x += eta d, end the solve
  static constexpr int NQ = 1;
  int64_t n;
  cx<R>* x;
  const cx<R>* d;
  cx<R> eta;
  __device__ __forceinline__ bool skip(const SolveState* st) const { return st->half == 0; }
  __device__ __forceinline__ void load(const SolveState* st) { eta = narrow<R>(st->eta); }
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) { x[i] = cadd(x[i], cmul(eta, d[i])); }
  __device__ void finish(const double*, SolveState* st) { st->poll.done = 1; }
};
template <class R> struct TqU : PhaseBase {  // u = w + beta u_{m+1}; v = beta A u_{m+1} + beta^2 v
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* w;
  const cx<R>* un;
  const cx<R>* uh;
  cx<R>* u;
  cx<R>* v;
  cx<R> beta, beta2;
  __device__ __forceinline__ bool skip(const SolveState* st) const { return st->half != 0; }
  __device__ __forceinline__ void load(const SolveState* st) {
    beta = narrow<R>(st->beta);
    beta2 = cmul(beta, beta);
  }
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) {
    u[i] = cadd(w[i], cmul(beta, un[i]));
    v[i] = cadd(cmul(beta, uh[i]), cmul(beta2, v[i]));
  }
  __device__ void finish(const double*, SolveState*) {}
};

// ---------------------------------------------------------------------------
// BiCGstab(l) (Sleijpen-Fokkema, vanilla; Sec. 3.1): l BiCG steps on
// r^_0..r^_l, u^_0..u^_l, then the minimal-residual update of degree l.  The
// minimal-residual coefficients come from the Gram matrix of r^_0..r^_l
// (one pass, every pair reduced at once) by a complex Cholesky solve of the
// normal equations in one thread: in exact arithmetic the same solution as
// modified Gram-Schmidt on the vectors, with one pass instead of l(l+1)/2.
// With the coefficients g_j in the original vectors the update is
//   x += sum_j g_j r^_{j-1},  r^_0 -= sum_j g_j r^_j,  u^_0 -= sum_j g_j u^_j.
// ---------------------------------------------------------------------------
struct BlVecs {
  void* rh[kMaxEll + 1];
  void* uh[kMaxEll + 1];
};
template <class R> struct BlRho : PhaseBase {  // rho1 = <r~, r^_j>; beta = alpha rho1 / rho0 (cycle start: rho0 = -omega rho0)
  static constexpr int NQ = 2;
  int64_t n;
  MvOut<R> mv;
  cx<R>* out;        // r^_j when mv holds partial sums
  const cx<R>* rt;
  bool start;
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> v = mv.get(i);
    if (mv.P) out[i] = v;
    acc_dotc(acc, rt[i], v);
  }
  __device__ void finish(const double* t, SolveState* st) {
    if (start) st->rho_old = cmul(cscale(-1.0, st->omega), st->rho_old);
    if (tiny<R>(st->rho_old)) { set_breakdown(st, CCG_BD_RHO); return; }
    const double2 rho1 = mkc(t[0], t[1]);
    st->beta = cdiv(cmul(st->alpha, rho1), st->rho_old);
    st->rho_old = rho1;
  }
};
template <class R> struct BlU : PhaseBase {  // u^_i = r^_i - beta u^_i, i <= j
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  BlVecs vv;
  int j;
  cx<R> beta;
  __device__ __forceinline__ void load(const SolveState* st) { beta = narrow<R>(st->beta); }
  template <class A> __device__ __forceinline__ void element(int64_t e, A*) {
    for (int i = 0; i <= j; ++i) {
      const cx<R>* ri = static_cast<const cx<R>*>(vv.rh[i]);
      cx<R>* ui = static_cast<cx<R>*>(vv.uh[i]);
      ui[e] = csub(ri[e], cmul(beta, ui[e]));
    }
  }
  __device__ void finish(const double*, SolveState*) {}
};
template <class R> struct BlGamma : PhaseBase {  // u^_{j+1} = A u^_j; gamma = <r~, u^_{j+1}>, alpha = rho0 / gamma
  static constexpr int NQ = 2;
  int64_t n;
  MvOut<R> mv;
  cx<R>* out;
  const cx<R>* rt;
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> v = mv.get(i);
    if (mv.P) out[i] = v;
    acc_dotc(acc, rt[i], v);
  }
  __device__ void finish(const double* t, SolveState* st) {
    const double2 g = mkc(t[0], t[1]);
    if (tiny<R>(g)) { set_breakdown(st, CCG_BD_SIGMA); return; }
    st->alpha = cdiv(st->rho_old, g);
  }
};
template <class R> struct BlR : PhaseBase {  // r^_i -= alpha u^_{i+1}, i <= j; x += alpha u^_0; ||r^_0||
  static constexpr int NQ = 1;
  int64_t n;
  BlVecs vv;
  int j;
  cx<R>* x;
  cx<R> alpha;
  __device__ __forceinline__ void load(const SolveState* st) { alpha = narrow<R>(st->alpha); }
  template <class A> __device__ __forceinline__ void element(int64_t e, A* acc) {
    const cx<R>* u0 = static_cast<const cx<R>*>(vv.uh[0]);
    x[e] = cadd(x[e], cmul(alpha, u0[e]));
    for (int i = 0; i <= j; ++i) {
      cx<R>* ri = static_cast<cx<R>*>(vv.rh[i]);
      const cx<R>* ui1 = static_cast<const cx<R>*>(vv.uh[i + 1]);
      const cx<R> v = csub(ri[e], cmul(alpha, ui1[e]));
      ri[e] = v;
      if (i == 0) acc_nrm2(acc, v);
    }
  }
  __device__ void finish(const double* t, SolveState* st) {  // a BiCG step may end the solve
    const double rel = sqrt(t[0]) / st->poll.ynorm;
    const int status = nonfinite(rel) ? ST_NONFINITE : (rel <= st->tol ? ST_OK : -100);
    if (status == -100) return;
    const int k = st->poll.k + 1;
    st->poll.k = k;
    st->poll.relres = rel;
    st->hist[k] = rel;
    st->poll.status = status;
    st->poll.done = 1;
  }
};
// Gram matrix of r^_0..r^_L (r^_L from the product just made): the pairs
// (i, j) with 1 <= i <= j <= L and (i, 0); then the normal equations.
template <class R, int L> struct BlGram : PhaseBase {
  static constexpr int NP = L * (L + 1) / 2 + L;
  static constexpr int NQ = 2 * NP;
  int64_t n;
  MvOut<R> mv;
  BlVecs vv;
  template <class A> __device__ __forceinline__ void element(int64_t e, A* acc) {
    cx<R> r[L + 1];
#pragma unroll
    for (int i = 0; i < L; ++i) r[i] = static_cast<const cx<R>*>(vv.rh[i])[e];
    r[L] = mv.get(e);
    if (mv.P) static_cast<cx<R>*>(vv.rh[L])[e] = r[L];
    int q = 0;
#pragma unroll
    for (int i = 1; i <= L; ++i) {
#pragma unroll
      for (int j = i; j <= L; ++j) { acc_dotc(acc + 2 * q, r[i], r[j]); ++q; }
      acc_dotc(acc + 2 * q, r[i], r[0]);
      ++q;
    }
  }
  __device__ void finish(const double* t, SolveState* st) {
    double2 M[L][L], b[L];
    int q = 0;
    for (int i = 0; i < L; ++i) {
      for (int j = i; j < L; ++j) {
        M[i][j] = mkc(t[2 * q], t[2 * q + 1]);
        M[j][i] = cconj(M[i][j]);
        ++q;
      }
      b[i] = mkc(t[2 * q], t[2 * q + 1]);
      ++q;
    }
    // M = C C^H (C lower triangular), then C c = b, C^H g = c
    double2 Cm[L][L];
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j) Cm[i][j] = mkc(0.0, 0.0);
    for (int j = 0; j < L; ++j) {
      double d = M[j][j].x;
      for (int k = 0; k < j; ++k) d -= Cm[j][k].x * Cm[j][k].x + Cm[j][k].y * Cm[j][k].y;
      if (!(d > tiny_guard<R>() * M[j][j].x) || tiny<R>(d)) { set_breakdown(st, CCG_BD_MU); return; }
      const double cjj = sqrt(d);
      Cm[j][j] = mkc(cjj, 0.0);
      for (int i = j + 1; i < L; ++i) {
        double2 s = M[i][j];
        for (int k = 0; k < j; ++k) s = csub(s, cmul(Cm[i][k], cconj(Cm[j][k])));
        Cm[i][j] = cscale(1.0 / cjj, s);
      }
    }
    double2 c[L], g[L];
    for (int i = 0; i < L; ++i) {
      double2 s = b[i];
      for (int k = 0; k < i; ++k) s = csub(s, cmul(Cm[i][k], c[k]));
      c[i] = cscale(1.0 / Cm[i][i].x, s);
    }
    for (int i = L - 1; i >= 0; --i) {
      double2 s = c[i];
      for (int k = i + 1; k < L; ++k) s = csub(s, cmul(cconj(Cm[k][i]), g[k]));
      g[i] = cscale(1.0 / Cm[i][i].x, s);
    }
    for (int i = 0; i < L; ++i) st->bl_g[i] = g[i];
    st->omega = g[L - 1];
  }
};
template <class R> struct BlMR : PhaseBase {  // the minimal-residual update; ||r^_0||, <r~, r^_0>
  static constexpr int NQ = 3;
  int64_t n;
  BlVecs vv;
  int L;
  cx<R>* x;
  const cx<R>* rt;
  cx<R> g[kMaxEll];
  __device__ __forceinline__ void load(const SolveState* st) {
    for (int i = 0; i < L; ++i) g[i] = narrow<R>(st->bl_g[i]);
  }
  template <class A> __device__ __forceinline__ void element(int64_t e, A* acc) {
    cx<R> xe = x[e];
    cx<R>* r0 = static_cast<cx<R>*>(vv.rh[0]);
    cx<R>* u0 = static_cast<cx<R>*>(vv.uh[0]);
    cx<R> r0e = r0[e], u0e = u0[e];
    const cx<R> r0_old = r0e;
    for (int j = 1; j <= L; ++j) {
      const cx<R> rprev = j == 1 ? r0_old : static_cast<const cx<R>*>(vv.rh[j - 1])[e];
      xe = cadd(xe, cmul(g[j - 1], rprev));
      r0e = csub(r0e, cmul(g[j - 1], static_cast<const cx<R>*>(vv.rh[j])[e]));
      u0e = csub(u0e, cmul(g[j - 1], static_cast<const cx<R>*>(vv.uh[j])[e]));
    }
    x[e] = xe;
    r0[e] = r0e;
    u0[e] = u0e;
    acc_nrm2(acc, r0e);
    acc_dotc(acc + 1, rt[e], r0e);
  }
  __device__ void finish(const double* t, SolveState* st) {
    if (end_iteration(st, st->poll.k + 1, sqrt(t[0]) / st->poll.ynorm, 0)) return;
    if (tiny<R>(st->omega)) { set_breakdown(st, CCG_BD_OMEGA); return; }
    // start of the next cycle: rho0 = -omega rho0, then step 0's rho1 and beta
    st->rho_old = cmul(cscale(-1.0, st->omega), st->rho_old);
    if (tiny<R>(st->rho_old)) { set_breakdown(st, CCG_BD_RHO); return; }
    const double2 rho1 = mkc(t[1], t[2]);
    st->beta = cdiv(cmul(st->alpha, rho1), st->rho_old);
    st->rho_old = rho1;
  }
};
template <class R> struct ZeroVec : PhaseBase {
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  cx<R>* v;
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) { v[i] = mk<R>(0, 0); }
  __device__ void finish(const double*, SolveState*) {}
};

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
struct GmBuf {
  double2* H;             // (m + 1) x m Hessenberg matrix, H[i * m + j]
  double2* g;             // m + 1: the rotated right-hand side
  double* cs;             // m rotation cosines
  double2* sn;            // m rotation sines
  double2* h2;            // m + 1: the second projection of the step
  double2* yv;            // m: the least-squares solution of the cycle
  double2* part;          // grid x (m + 1) per-block partial sums
  unsigned int* counter;  // arrival counter of the passes, 0 between them
  int m;
};

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

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Warps per matrix row in the row sweep (gemv_n_rows).
constexpr int kRowSplit = 4;

// Launch geometry of the dense sweeps for one operator.
// Resident blocks per SM of the column-tiled sweep (A^H x alone, or A x1 with
// A^H x2), from the occupancy calculator.
template <class R> static int tile_occupancy(int unit, bool both) {
  static int cache[2][2] = {{0, 0}, {0, 0}};
  int& c = cache[unit == 2 ? 1 : 0][both ? 1 : 0];
  if (c == 0) {
    const void* fn = nullptr;
    if constexpr (sizeof(R) == 4) {
      if (unit == 2) fn = both ? (const void*)gemv_tile<R, 2, 4, true, true> : (const void*)gemv_tile_h<R, 2, 4>;
      else fn = both ? (const void*)gemv_tile<R, 1, 4, true, true> : (const void*)gemv_tile_h<R, 1, 4>;
    } else {
      fn = both ? (const void*)gemv_tile<R, 1, 4, true, true> : (const void*)gemv_tile_h<R, 1, 4>;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kBlock, 0) != cudaSuccess) {
      cudaGetLastError();
      occ = 2;
    }
    c = std::max(1, occ);
  }
  return c;
}

// Row ranges of a column-tiled sweep: enough (column chunk, row range)
// blocks to fill every SM once at the kernel's occupancy.
struct TileSplit {
  int nsplit;
  int64_t rows_per_range;
};
static TileSplit tile_split(int64_t n, int ncb, int64_t target) {
  int64_t ns = (target + ncb - 1) / ncb;
  ns = std::max<int64_t>(1, std::min<int64_t>(ns, std::min<int64_t>(32, (n + kWarps - 1) / kWarps)));
  TileSplit t;
  t.rows_per_range = (n + ns - 1) / ns;
  t.nsplit = (int)((n + t.rows_per_range - 1) / t.rows_per_range);
  return t;
}

template <class R> struct Dense {
  const cx<R>* A;
  int64_t lda, n;
  int unit;
  int grid_rows;            // gemv_n_rows blocks
  int ncb;                  // gemv_tile column chunks
  TileSplit tc, tb;         // row ranges for A^H x, and for A x1 with A^H x2
  static constexpr int E = 4;

  Dense(const ccg_operator* op, int num_sms) {
    A = static_cast<const cx<R>*>(op->A);
    lda = op->lda;
    n = op->n;
    unit = op->unit;
    const int64_t rows_blocks = (n + kWarps - 1) / kWarps;
    grid_rows = (int)std::min<int64_t>((n + kWarps / kRowSplit - 1) / (kWarps / kRowSplit), 1 << 30);
    (void)rows_blocks;
    const int64_t nunits = n / unit;
    ncb = (int)((nunits + 32 * E - 1) / (32 * E));
    dense = op->kind == CCG_OPK_DENSE;
    if (dense) {
      tc = tile_split(n, ncb, (int64_t)num_sms * tile_occupancy<R>(unit, false));
      tb = tile_split(n, ncb, (int64_t)num_sms * tile_occupancy<R>(unit, true));
    } else {
      tc = tb = TileSplit{1, n};
    }
    dip_bytes = op->dip.sweep_bytes;
  }
  bool dense = true;
  double dip_bytes = 0.0;
  size_t p1_elems() const { return dense ? (size_t)ncb * n : 0; }
  size_t p2_elems() const { return dense ? (size_t)std::max(tc.nsplit, tb.nsplit) * n : 0; }
  double sweep_bytes() const { return dense ? (double)n * (double)n * sizeof(cx<R>) : dip_bytes; }
};

// Rows per thread and grid of the GMRES orthogonalisation passes.
static int gm_rows_per_thread(int64_t n) {
  return n <= (int64_t)kBlock * 1024 ? 1 : (n <= (int64_t)kBlock * 2048 ? 2 : (n <= (int64_t)kBlock * 4096 ? 4 : 8));
}
static int gm_grid(int64_t n) {
  const int64_t per = (int64_t)kBlock * gm_rows_per_thread(n);
  return (int)std::max<int64_t>(1, (n + per - 1) / per);
}
static int64_t gm_ldv(int64_t n) { return (n + 63) / 64 * 64; }

template <class R> struct Ws {
  cx<R>* vec[12];
  cx<R>* basis;     // GMRES: m + 1 vectors, leading dimension ldv
  int64_t ldv;
  GmBuf gm;
  cx<R>* P1;
  cx<R>* P2;
  cx<R>* ystage;
  cx<R>* xstage;
  double* partials;
  unsigned int* counter;
  SolveState* st;
  double* hist;
  double* scratch;  // a few doubles for standalone results
};

// basis = m + 1 GMRES basis vectors (0 for the other methods).
template <class R> static size_t ws_bytes(int64_t n, const Dense<R>& d, int maxit, int basis = 0) {
  size_t b = 0;
  if (basis > 0) {
    const int m = basis - 1;
    b += align256((size_t)basis * gm_ldv(n) * sizeof(cx<R>));
    b += align256((size_t)(m + 1) * m * sizeof(double2)) + 4 * align256((size_t)(m + 1) * sizeof(double2)) +
         align256((size_t)m * sizeof(double));
    b += align256((size_t)gm_grid(n) * (m + 1) * sizeof(double2)) + align256(counter_words(gm_grid(n)) * sizeof(unsigned int));
  }
  b += 12 * align256(n * sizeof(cx<R>));
  b += align256(std::max(d.p1_elems(), d.p2_elems()) * sizeof(cx<R>));
  b += align256(d.p2_elems() * sizeof(cx<R>));
  b += 2 * align256(n * sizeof(cx<R>));
  b += align256(kMaxRedBlocks * kMaxNQ * sizeof(double));
  b += align256(sizeof(unsigned int));
  b += align256(sizeof(SolveState));
  b += align256((size_t)(maxit + 1) * sizeof(double));
  b += align256(16 * sizeof(double));
  return b;
}

template <class R> static Ws<R> ws_carve(char* base, int64_t n, const Dense<R>& d, int maxit, int basis = 0) {
  Ws<R> w;
  size_t off = 0;
  auto take = [&](size_t bytes) { char* p = base + off; off += align256(bytes); return p; };
  w.basis = nullptr;
  w.ldv = gm_ldv(n);
  std::memset(&w.gm, 0, sizeof(w.gm));
  if (basis > 0) {
    const int m = basis - 1;
    w.basis = reinterpret_cast<cx<R>*>(take((size_t)basis * w.ldv * sizeof(cx<R>)));
    w.gm.H = reinterpret_cast<double2*>(take((size_t)(m + 1) * m * sizeof(double2)));
    w.gm.g = reinterpret_cast<double2*>(take((size_t)(m + 1) * sizeof(double2)));
    w.gm.sn = reinterpret_cast<double2*>(take((size_t)(m + 1) * sizeof(double2)));
    w.gm.h2 = reinterpret_cast<double2*>(take((size_t)(m + 1) * sizeof(double2)));
    w.gm.yv = reinterpret_cast<double2*>(take((size_t)(m + 1) * sizeof(double2)));
    w.gm.cs = reinterpret_cast<double*>(take((size_t)m * sizeof(double)));
    w.gm.part = reinterpret_cast<double2*>(take((size_t)gm_grid(n) * (m + 1) * sizeof(double2)));
    w.gm.counter = reinterpret_cast<unsigned int*>(take(counter_words(gm_grid(n)) * sizeof(unsigned int)));
    w.gm.m = m;
  }
  for (int i = 0; i < 12; ++i) w.vec[i] = reinterpret_cast<cx<R>*>(take(n * sizeof(cx<R>)));
  w.P1 = reinterpret_cast<cx<R>*>(take(std::max(d.p1_elems(), d.p2_elems()) * sizeof(cx<R>)));
  w.P2 = reinterpret_cast<cx<R>*>(take(d.p2_elems() * sizeof(cx<R>)));
  w.ystage = reinterpret_cast<cx<R>*>(take(n * sizeof(cx<R>)));
  w.xstage = reinterpret_cast<cx<R>*>(take(n * sizeof(cx<R>)));
  w.partials = reinterpret_cast<double*>(take(kMaxRedBlocks * kMaxNQ * sizeof(double)));
  w.counter = reinterpret_cast<unsigned int*>(take(sizeof(unsigned int)));
  w.st = reinterpret_cast<SolveState*>(take(sizeof(SolveState)));
  w.hist = reinterpret_cast<double*>(take((size_t)(maxit + 1) * sizeof(double)));
  w.scratch = reinterpret_cast<double*>(take(16 * sizeof(double)));
  return w;
}

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
    // One element per thread up to about 2.7 blocks per SM: on large
    // systems fewer, longer-running blocks leave less to the cross-block
    // reduction (measured on the 412k-unknown dipole system: 405 blocks beat
    // 1216 by 7%; n = 8192 keeps its 32 blocks)
    const int64_t per_block = (int64_t)kBlock * h->phase_elems;
    grid_vec = (int)std::min<int64_t>((d.n + per_block - 1) / per_block, (int64_t)h->num_sms * 8 / 3);
    grid_vec = std::max(1, std::min(grid_vec, kMaxRedBlocks));
  }

  template <class P> void phase(const P& p) {
    phase_kernel<P, acc_t<R>><<<grid_vec, kBlock, 0, s>>>(p, w.st, red);
    ++h->launches;
  }

  MvOut<R> plain(const cx<R>* y) const { MvOut<R> m; m.y = y; m.P = nullptr; m.ld = d.n; m.nparts = 1; return m; }

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
      dipole_apply(op, x, y, false, st, s, rec);
      h->launches += op->dip.kernels;
    } else {
      if constexpr (sizeof(R) == 4) {
        if (d.unit == 2)
          gemv_n_rows<R, 2, kRowSplit><<<d.grid_rows, kBlock, 0, s>>>(d.A, d.lda, d.n, x, y, st, rec);
        else
          gemv_n_rows<R, 1, kRowSplit><<<d.grid_rows, kBlock, 0, s>>>(d.A, d.lda, d.n, x, y, st, rec);
      } else {
        gemv_n_rows<R, 1, kRowSplit><<<d.grid_rows, kBlock, 0, s>>>(d.A, d.lda, d.n, x, y, st, rec);
      }
      ++h->launches;
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
      dipole_apply(op, x, y, true, st, s, rec);
      h->launches += op->dip.kernels;
      timing_end(h, kDt, CCG_SWEEP_C, d.sweep_bytes());
      return plain(y);
    }
    dim3 grid(d.ncb, d.tc.nsplit);
    const int64_t rpr = d.tc.rows_per_range;
    if constexpr (sizeof(R) == 4) {
      if (d.unit == 2)
        gemv_tile_h<R, 2, Dense<R>::E><<<grid, kBlock, 0, s>>>(d.A, d.lda, d.n, rpr, x, w.P2, st, rec);
      else
        gemv_tile_h<R, 1, Dense<R>::E><<<grid, kBlock, 0, s>>>(d.A, d.lda, d.n, rpr, x, w.P2, st, rec);
    } else {
      gemv_tile_h<R, 1, Dense<R>::E><<<grid, kBlock, 0, s>>>(d.A, d.lda, d.n, rpr, x, w.P2, st, rec);
    }
    ++h->launches;
    timing_end(h, kDt, CCG_SWEEP_C, d.sweep_bytes());
    MvOut<R> m; m.y = nullptr; m.P = w.P2; m.ld = d.n; m.nparts = d.tc.nsplit;
    return m;
  }
  // A x1 and A^H x2: dense operators from one sweep (ncb partials in P1,
  // nsplit in P2); others by two applications into y1, y2.
  void apply_both(const cx<R>* x1, const cx<R>* x2, cx<R>* y1, cx<R>* y2, MvOut<R>& o1, MvOut<R>& o2,
                  const SolveState* st) {
    if (op->kind != CCG_OPK_DENSE) {
      o1 = apply_n(x1, y1, st);
      o2 = apply_c(x2, y2, st);
      return;
    }
    dim3 grid(d.ncb, d.tb.nsplit);
    const int64_t rpr = d.tb.rows_per_range;
    timing_begin(h);
    int* rec = timing_rec(h);
    if constexpr (sizeof(R) == 4) {
      if (d.unit == 2)
        gemv_tile<R, 2, Dense<R>::E, true, true><<<grid, kBlock, 0, s>>>(d.A, d.lda, d.n, rpr, x1, x2, w.P1, w.P2, st, rec);
      else
        gemv_tile<R, 1, Dense<R>::E, true, true><<<grid, kBlock, 0, s>>>(d.A, d.lda, d.n, rpr, x1, x2, w.P1, w.P2, st, rec);
    } else {
      gemv_tile<R, 1, Dense<R>::E, true, true><<<grid, kBlock, 0, s>>>(d.A, d.lda, d.n, rpr, x1, x2, w.P1, w.P2, st, rec);
    }
    ++h->launches;
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
  int rc = arena_reserve(h, ws_bytes<R>(n, dl, maxit, basis));
  if (rc != CCG_OK) return rc;
  Ws<R> w = ws_carve<R>(h->arena, n, dl, maxit, basis);
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
  if ((rc = solve_core<R>(h, method, op, w, y, x, tol, maxit, false, &fin)) != CCG_OK) return rc;
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
struct RefResid : PhaseBase {  // r = y - A x (double); r32 = round(r); d32 = 0
  static constexpr int NQ = 3;   // ||y||^2, ||r||^2, non-finite count in y
  int64_t n;
  const double2* y;
  MvOut<double> ax;
  float2* r32;
  float2* d32;
  int outer;
  bool ax_zero;
  __device__ __forceinline__ void load(const SolveState* st) { ax_zero = st->skip_mv != 0; }
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const double2 yi = y[i];
    const double2 ri = ax_zero ? yi : csub(yi, ax.get(i));
    r32[i] = make_float2((float)ri.x, (float)ri.y);
    d32[i] = make_float2(0.f, 0.f);
    acc[0] += yi.x * yi.x + yi.y * yi.y;
    acc[1] += ri.x * ri.x + ri.y * ri.y;
    if (!(isfinite(yi.x) && isfinite(yi.y))) acc[2] += 1.0;
  }
  __device__ void finish(const double* t, SolveState* st) {
    st->poll.k = outer;
    st->skip_mv = 0;
    if (t[2] != 0.0) { st->poll.status = ST_NONFINITE; st->poll.done = 1; return; }
    const double yn = sqrt(t[0]);
    st->poll.ynorm = yn;
    if (yn == 0.0) {
      st->zero_rhs = 1;
      st->hist[outer] = 0.0;
      st->poll.relres = 0.0;
      st->poll.status = ST_OK;
      st->poll.done = 1;
      return;
    }
    const double rel = sqrt(t[1]) / yn;
    st->hist[outer] = rel;
    st->poll.relres = rel;
    if (nonfinite(rel)) { st->poll.status = ST_NONFINITE; st->poll.done = 1; return; }
    if (rel <= st->tol) { st->poll.status = ST_OK; st->poll.done = 1; return; }
    if (outer >= st->maxit) { st->poll.status = ST_NOT_CONVERGED; st->poll.done = 1; }
  }
};
struct RefUpdate : PhaseBase {  // x += widen(d32)
  static constexpr bool kReduce = false;
  static constexpr int NQ = 1;
  int64_t n;
  double2* x;
  const float2* d32;
  template <class A> __device__ __forceinline__ void element(int64_t i, A*) {
    const float2 d = d32[i];
    x[i] = cadd(x[i], make_double2((double)d.x, (double)d.y));
  }
  __device__ void finish(const double*, SolveState*) {}
};

int solve_refined(ccg_handle* h, int method, const ccg_operator* op, const ccg_operator* op_in, const void* y_in,
                  void* x_in, double tol, int max_outer, double inner_tol, int inner_maxit, double* res_hist,
                  int* inner_iters, ccg_info* info) {
  const int64_t n = op->n;
  Dense<double> d64(op, h->num_sms);
  Dense<float> d32(op_in, h->num_sms);
  const size_t b64 = ws_bytes<double>(n, d64, max_outer);
  const int basis = method == M_GMRES ? h->gm_restart + 1 : 0;
  int rc = arena_reserve(h, b64 + ws_bytes<float>(n, d32, inner_maxit, basis));
  if (rc != CCG_OK) return rc;
  Ws<double> w = ws_carve<double>(h->arena, n, d64, max_outer);
  Ws<float> wi = ws_carve<float>(h->arena + b64, n, d32, inner_maxit, basis);
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
    if ((rc = solve_core<float>(h, method, op_in, wi, r32, dd, inner_tol, inner_maxit, true, &fin)) != CCG_OK)
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
