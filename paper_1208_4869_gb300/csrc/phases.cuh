// Fused update kernels of the Krylov iterations ("phases"): each struct is
// one method step's elementwise updates and dot products over the vectors
// (element), and the scalar recurrences its reduced sums feed (finish).
// They run as single kernels (phase_kernel, the multi-kernel solve loop of
// solve.cu) or as steps of the persistent solve (persist.cu).  Methods: the
// Sec. 2.1 PIM set (BiCGSTAB, CGNR, QMR, BiCG, CGS, CGNE, TFQMR), the Sec. 2.2
// complex-symmetric CG, BiCGstab(l) (Sec. 3.1) and COCR (Sec. 3.4).
#pragma once

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
  pdl_wait();
  pdl_launch();
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
  pdl_wait();
  pdl_launch();
  int mine = 0;
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
    const cx<R> v = x[i];
    mine |= (v.x != (R)0 || v.y != (R)0);
  }
  if (__syncthreads_or(mine) && threadIdx.x == 0) st->skip_mv = 0;
}

// Whether the start vector is zero (persistent solve): skip_mv = 1 when every
// entry of x is zero, so the product A x0 is not formed.
template <class R> struct XNz : PhaseBase {
  static constexpr int NQ = 1;
  int64_t n;
  const cx<R>* x;
  template <class A> __device__ __forceinline__ void element(int64_t i, A* acc) {
    const cx<R> v = x[i];
    if (v.x != (R)0 || v.y != (R)0) acc_add1(acc[0]);
  }
  __device__ void finish(const double* t, SolveState* st) { st->skip_mv = t[0] == 0.0 ? 1 : 0; }
};

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
// Mixed-precision refinement: r = y - A x and x += d in complex128 around a
// complex64 inner solve of A d = r.
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


}  // namespace ccg
