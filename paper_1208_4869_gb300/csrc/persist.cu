// Persistent solves: the whole Krylov iteration of one dense system, or of
// many dense systems of different sizes, in one cooperative launch.
//
// The grid (every resident block of the GPU) is cut into groups, one per
// system, sized by the system's share of the matrix bytes.  A group runs its
// system's method exactly as the multi-kernel loop of solve.cu does -- the
// same phase structs (phases.cuh) and sweep bodies (gemv.cuh) -- but with a
// group barrier where that loop ends a kernel: vector phases stride over the
// group's blocks, their sums meet in the group's last block to arrive (which
// forms the method's scalars, as a phase kernel's last block does), and
// sweeps take row blocks or (column chunk, row range) tiles in turn.  Groups
// never wait for one another, so systems of different sizes and iteration
// counts advance independently inside one launch.
//
// Barriers count arrivals on one word per group and spin with a bounded
// wait: after `limit` SM clock cycles a block gives up, raises the launch's
// fault flag and leaves, and the host returns CCG_ERR_TIMEOUT.  A test hook
// withholds one block's arrival to exercise that path (CCG_OPT_TEST_WITHHOLD).
//
// Vectors are rewritten between sweeps inside the launch, so sweeps read them
// with coherent loads (KC = true); the barrier's acquire orders those reads
// after the writes of every block of the group.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "reduce.cuh"
#include "gemv.cuh"
#include "phases.cuh"
#include "workspace.cuh"
#include "fx.cuh"
#include "tune_table.h"
#include "internal.h"

namespace ccg {

// ---------------------------------------------------------------------------
// Group barrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// All G blocks of a group meet at their epoch-th barrier (epoch counted by
// each block, the same sequence in every block of the group): a block adds 1
// to the group's arrival count with release semantics, without waiting for
// the result, then polls the count with acquire loads until it reaches
// epoch x G -- one L2 round trip per block instead of an arrival, a last
// arriver's release and the waiters' observation of it.  The count only
// grows during a launch (it is zeroed before), and the comparison is
// modular.  False if this block gave up after `limit` clock cycles (it then
// raises *fault) or another block already raised it.
__device__ __forceinline__ bool group_sync(GroupBar* b, int G, unsigned& epoch, long long limit, int* fault) {
  __shared__ int ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    int good = 1;
    if (G > 1) {
      red_release_add_u32(&b->count, 1u);
      const unsigned target = epoch * (unsigned)G;
      if ((int)(ld_acquire_u32(&b->count) - target) < 0) {
        const long long t0 = clock64();
        while ((int)(ld_acquire_u32(&b->count) - target) < 0) {
          if (clock64() - t0 > limit) {
            good = 0;
            atomicExch(fault, 1);
            break;
          }
        }
      }
    } else {
      __threadfence();
    }
    if (good && ld_relaxed_s32(fault)) good = 0;
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// ---------------------------------------------------------------------------
// One system's group.
// ---------------------------------------------------------------------------
template <class R, int U> struct PkCtx {
  const PkSys<R>& S;
  int lb, G;
  long long limit;
  int* fault;
  Red red;
  cx<R>* tsm;  // shared memory of the tile sweeps
  int nsw = 0; // sweeps so far (the parity picks the fixed-point sweep's exponent slot)
  unsigned epoch = 0;  // barriers passed

  __device__ PkCtx(const PkSys<R>& s, int lb_, int G_, long long lim, int* f, cx<R>* sm)
      : S(s), lb(lb_), G(G_), limit(lim), fault(f), tsm(sm) {
    red.partials = s.partials;
    red.counter = s.counter;
  }
  // Barrier, then: does the solve go on?
  __device__ __forceinline__ bool sync() {
    if (!group_sync(S.bar, G, epoch, limit, fault)) return false;
    return *reinterpret_cast<volatile const int*>(&S.st->poll.done) == 0;
  }
  // A vector phase is cut into the same `nvb` virtual blocks as the phase
  // kernel of the kernel-per-step loop (its grid), each reduced on its own
  // and summed in virtual-block order, so the sums -- and the whole solve --
  // are bitwise those of that loop, whatever the group's size.  A group
  // block takes virtual blocks lb, lb + G, ...; blocks beyond nvb go on to
  // the barrier.
  template <class P> __device__ __forceinline__ void phase(P& p) {
    const int nvb = S.nvb;
    if (lb >= nvb) return;
    SolveState* st = S.st;
    if (p.skip(st)) return;
    p.load(st);
    const int64_t stride = (int64_t)nvb * kBlock;
    for (int vb = lb; vb < nvb; vb += G) {
      acc_t<R> acc[P::NQ];
#pragma unroll
      for (int q = 0; q < P::NQ; ++q) acc_zero(acc[q]);
      for (int64_t i = (int64_t)vb * kBlock + threadIdx.x; i < p.n; i += stride) p.element(i, acc);
      if (P::kReduce) {
        double tot[P::NQ];
        if (group_reduce<P::NQ>(acc, red.partials, red.counter, tot, vb, nvb) && threadIdx.x == 0) p.finish(tot, st);
      }
    }
  }
  __device__ __forceinline__ void count_sweep() {
    if (lb == 0 && threadIdx.x == 0) S.st->sweeps += 1;
  }
  __device__ __forceinline__ MvOut<R> plain(const cx<R>* y) const {
    MvOut<R> m;
    m.y = y; m.P = nullptr; m.ld = S.n; m.nparts = 1;
    return m;
  }
  // y = A x
  __device__ MvOut<R> sweep_n(const cx<R>* x, cx<R>* y) {
    if constexpr (sizeof(R) == 8) {
      if (S.fxC != nullptr) {
        fx_sweep(x, y);
        count_sweep();
        return plain(y);
      }
    }
    gemv_rows_body<R, U, kRowSplit, true>(S.A, S.lda, S.n, x, y, lb, G);
    count_sweep();
    return plain(y);
  }
  // The group's fixed-point digits of x1 into xd1 and of the row-scaled x2
  // into xd2 (either may be null), with their exponents -- the loop's
  // fx_split_vector across the group's blocks: the largest exponents meet in
  // the sweep's pair of exponent words (two pairs alternate between sweeps;
  // block 0 clears the other pair, last read two barriers ago), then each
  // block writes its share of the digits.  bad: an operand is not finite (the
  // sweep then takes the FP64 pipe).  False if a barrier gave up.
  __device__ bool fx_split_group(const double2* x1, int4* xd1, const double2* x2, int4* xd2, int& e1, int& e2,
                                 bool& bad) {
    __shared__ int wm[2][kWarps];
    int* pair = S.fxe + 2 * (nsw & 1);
    int* other = S.fxe + 2 * ((nsw & 1) ^ 1);
    ++nsw;
    const int fm = max(S.fxrow[S.n + 1], 1);
    int m1 = 0, m2 = 0;
    const int64_t stride = (int64_t)G * kBlock;
    for (int64_t i = (int64_t)lb * kBlock + threadIdx.x; i < S.n; i += stride) {
      if (x1) {
        const double2 v = ldc_unit(x1 + i);
        m1 = max(m1, max(fx_exp(v.x), fx_exp(v.y)));
      }
      if (x2) {
        const double2 v = fx_row_scaled(ldc_unit(x2 + i), S.fxrow[i], fm);
        m2 = max(m2, max(fx_exp(v.x), fx_exp(v.y)));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m1 = max(m1, __shfl_xor_sync(0xffffffffu, m1, o));
      m2 = max(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    if ((threadIdx.x & 31) == 0) {
      wm[0][threadIdx.x >> 5] = m1;
      wm[1][threadIdx.x >> 5] = m2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int w = 1; w < kWarps; ++w) {
        m1 = max(m1, wm[0][w]);
        m2 = max(m2, wm[1][w]);
      }
      if (x1) atomicMax(pair, m1);
      if (x2) atomicMax(pair + 1, m2);
      if (lb == 0) {
        atomicExch(other, 0);
        atomicExch(other + 1, 0);
      }
    }
    if (!group_sync(S.bar, G, epoch, limit, fault)) return false;
    e1 = *reinterpret_cast<volatile const int*>(pair);
    e2 = *reinterpret_cast<volatile const int*>(pair + 1);
    bad = S.fxrow[S.n] != 0 || (x1 && e1 == 0x7FF) || (x2 && e2 == 0x7FF);
    if (!bad) {
      for (int64_t i = (int64_t)lb * kBlock + threadIdx.x; i < S.n; i += stride) {
        int4 q;
        if (x1) {
          const double2 v = ldc_unit(x1 + i);
          fx_split(v.x, e1, q.x, q.y);
          fx_split(v.y, e1, q.z, q.w);
          xd1[i] = q;
        }
        if (x2) {
          const double2 v = fx_row_scaled(ldc_unit(x2 + i), S.fxrow[i], fm);
          fx_split(v.x, e2, q.x, q.y);
          fx_split(v.y, e2, q.z, q.w);
          xd2[i] = q;
        }
      }
    }
    return group_sync(S.bar, G, epoch, limit, fault);
  }
  // complex128 y = A x in fixed point: the digits of x, then the rows from
  // the operator's digits
  __device__ void fx_sweep(const double2* x, double2* y) {
    int e1 = 0, e2 = 0;
    bool bad = false;
    if (!fx_split_group(x, S.xfx, nullptr, nullptr, e1, e2, bad)) return;
    gemv_fx_rows_body<kFxSplit, true>(S.A, S.lda, S.fxC, S.fxrow, S.n, x, S.xfx, e1, bad, y, lb, G);
  }
  // A^H x as ns_c partial vectors in P2
  __device__ MvOut<R> sweep_c(const cx<R>* x) {
    const int64_t nt = (int64_t)S.ncb * S.ns_c;
    bool fx = false;
    if constexpr (sizeof(R) == 8) {
      if (S.fxC != nullptr) {
        int e1 = 0, e2 = 0;
        bool bad = false;
        if (fx_split_group(nullptr, nullptr, x, S.xfx2, e1, e2, bad)) {
          fx = !bad;
          if (fx)
            for (int64_t t = lb; t < nt; t += G)
              gemv_fx_tile_body<true>(S.fxC, S.fxrow, S.n, S.rpr_c, S.xfx2, e2, S.P2, t % S.ncb, t / S.ncb, tsm);
        } else {
          fx = true;  // a barrier gave up: the caller's next barrier returns
        }
      }
    }
    if (!fx)
      for (int64_t t = lb; t < nt; t += G)
        gemv_tile_body<R, U, 4, false, true, true>(S.A, S.lda, S.n, S.rpr_c, nullptr, x, nullptr, S.P2, t % S.ncb,
                                                   t / S.ncb, tsm);
    count_sweep();
    MvOut<R> m;
    m.y = nullptr; m.P = S.P2; m.ld = S.n; m.nparts = S.ns_c;
    return m;
  }
  // A x1 (ncb partials in P1) and A^H x2 (ns_b partials in P2) from one read
  // of A; complex128 on the integer pipe: the two sweeps, A x1 into y1 (as
  // the kernel loop does)
  __device__ void sweep_both(const cx<R>* x1, const cx<R>* x2, cx<R>* y1, MvOut<R>& o1, MvOut<R>& o2) {
    if constexpr (sizeof(R) == 8) {
      if (S.fxC != nullptr) {
        o1 = sweep_n(x1, y1);
        o2 = sweep_c(x2);
        return;
      }
    }
    const int64_t nt = (int64_t)S.ncb * S.ns_b;
    for (int64_t t = lb; t < nt; t += G)
      gemv_tile_body<R, U, 4, true, true, true>(S.A, S.lda, S.n, S.rpr_b, x1, x2, S.P1, S.P2, t % S.ncb, t / S.ncb,
                                                tsm);
    count_sweep();
    o1.y = nullptr; o1.P = S.P1; o1.ld = S.n; o1.nparts = S.ncb;
    o2.y = nullptr; o2.P = S.P2; o2.ld = S.n; o2.nparts = S.ns_b;
  }
};

// The method's start and iterations for one group; returns when the solve has
// stopped or a barrier gave up.  Vector slots as in solve_core.
template <class R, int U, int method> __device__ void pk_run_method(PkCtx<R, U>& c);

// One group: its method, then (when asked and nothing failed) the final
// true residual ||y - A x||^2.
template <class R, int U, int method> __device__ void pk_run_group(PkCtx<R, U>& c) {
  pk_run_method<R, U, method>(c);
  const PkSys<R>& S = c.S;
  if (!S.want_true || ld_relaxed_s32(c.fault)) return;
  // every block of the group left the iteration at the same barrier
  MvOut<R> ax = c.sweep_n(S.x, S.V[11]);
  if (!group_sync(S.bar, c.G, c.epoch, c.limit, c.fault)) return;
  TrueRes<R> tr;
  tr.n = S.n; tr.y = S.y; tr.out = S.scratch; tr.ax = ax;
  c.phase(tr);
}

template <class R, int U, int method> __device__ void pk_run_method(PkCtx<R, U>& c) {
  const PkSys<R>& S = c.S;
  const int64_t n = S.n;
  SolveState* st = S.st;
  cx<R>* const* V = S.V;
  cx<R>* x = S.x;

  if constexpr (method == M_REFRES) {
    if constexpr (sizeof(R) == 8) {
      if (S.outer > 0) {
        RefUpdate u;
        u.n = n; u.x = x; u.d32 = S.d32;
        c.phase(u);
        if (!group_sync(S.bar, c.G, c.epoch, c.limit, c.fault)) return;
      }
      MvOut<R> ax;
      ax.y = nullptr; ax.P = nullptr; ax.ld = n; ax.nparts = 0;
      if (S.outer == 0 && !S.x0_zero) {
        { XNz<R> z; z.n = n; z.x = x; c.phase(z); }
        if (!group_sync(S.bar, c.G, c.epoch, c.limit, c.fault)) return;
      }
      if (!*reinterpret_cast<volatile const int*>(&st->skip_mv)) {
        ax = c.sweep_n(x, V[0]);
        if (!group_sync(S.bar, c.G, c.epoch, c.limit, c.fault)) return;
      }
      RefResid rp;
      rp.n = n; rp.y = S.y; rp.r32 = S.r32; rp.d32 = S.d32; rp.outer = S.outer; rp.ax = ax;
      c.phase(rp);
      group_sync(S.bar, c.G, c.epoch, c.limit, c.fault);
    }
    return;
  }
  // r0 = y - A x0, with the product skipped when x0 is known or found zero
  MvOut<R> ax;
  ax.y = nullptr; ax.P = nullptr; ax.ld = n; ax.nparts = 0;
  if (!S.x0_zero) {
    { XNz<R> z; z.n = n; z.x = x; c.phase(z); }
    if (!group_sync(S.bar, c.G, c.epoch, c.limit, c.fault)) return;
    if (!*reinterpret_cast<volatile const int*>(&st->skip_mv)) {
      ax = c.sweep_n(x, V[11]);
      if (!group_sync(S.bar, c.G, c.epoch, c.limit, c.fault)) return;
    }
  }
  {
    InitR<R> p;
    p.n = n; p.y = S.y; p.r = V[0]; p.c1 = nullptr; p.c2 = nullptr; p.method = method; p.ax = ax;
    if constexpr (method == M_BICGSTAB || method == M_COCG) p.c1 = V[1];
    else if constexpr (method == M_QMR) { p.c1 = V[1]; p.c2 = V[2]; }
    c.phase(p);
    if (!c.sync()) return;
  }
  for (int it = 0; it <= st->maxit; ++it) {
    if constexpr (method == M_BICGSTAB) {
      cx<R>*r = V[0], *rh = V[1], *pv = V[2], *v = V[3], *sv = V[4], *t = V[5];
      { BiP<R> a; a.n = n; a.r = r; a.p = pv; a.v = v; c.phase(a); }
      if (!c.sync()) return;
      MvOut<R> mv = c.sweep_n(pv, v);
      if (!c.sync()) return;
      { BiSigma<R> b; b.n = n; b.v = v; b.rh = rh; b.mv = mv; c.phase(b); }
      if (!c.sync()) return;
      { BiS<R> e; e.n = n; e.r = r; e.v = v; e.s = sv; c.phase(e); }
      if (!c.sync()) return;
      MvOut<R> mt = c.plain(t);
      if (!*reinterpret_cast<volatile const int*>(&st->half)) {
        mt = c.sweep_n(sv, t);
        if (!c.sync()) return;
      }
      { BiOmega<R> f; f.n = n; f.t = t; f.s = sv; f.mv = mt; c.phase(f); }
      if (!c.sync()) return;
      { BiXR<R> g; g.n = n; g.x = x; g.r = r; g.p = pv; g.s = sv; g.t = t; g.rh = rh; c.phase(g); }
      if (!c.sync()) return;
    } else if constexpr (method == M_CGNR) {
      cx<R>*r = V[0], *z = V[1], *pv = V[2], *wv = V[3];
      if (it == 0) {
        MvOut<R> mz = c.sweep_c(r);
        if (!c.sync()) return;
        { CgZ<R> z0; z0.n = n; z0.z = z; z0.p = pv; z0.mv = mz; c.phase(z0); }
        if (!c.sync()) return;
      }
      MvOut<R> mw = c.sweep_n(pv, wv);
      if (!c.sync()) return;
      { CgAlpha<R> a; a.n = n; a.w = wv; a.mv = mw; c.phase(a); }
      if (!c.sync()) return;
      { CgXR<R> b; b.n = n; b.x = x; b.r = r; b.p = pv; b.w = wv; c.phase(b); }
      if (!c.sync()) return;
      MvOut<R> mz = c.sweep_c(r);
      if (!c.sync()) return;
      { CgZ<R> e; e.n = n; e.z = z; e.p = nullptr; e.mv = mz; c.phase(e); }
      if (!c.sync()) return;
      { CgP<R> f; f.n = n; f.z = z; f.p = pv; c.phase(f); }
      if (!c.sync()) return;
    } else if constexpr (method == M_QMR) {
      cx<R>*r = V[0], *vt = V[1], *wt = V[2], *v = V[3], *wv = V[4], *pv = V[5], *q = V[6], *pt = V[7], *u = V[8],
           *dv = V[9], *sv = V[10];
      if (it == 0) {
        { QVW<R> f; f.n = n; f.vt = vt; f.wt = wt; f.v = v; f.w = wv; c.phase(f); }
        if (!c.sync()) return;
      }
      { QPQ<R> a; a.n = n; a.v = v; a.w = wv; a.p = pv; a.q = q; c.phase(a); }
      if (!c.sync()) return;
      MvOut<R> m1, m2;
      c.sweep_both(pv, q, pt, m1, m2);
      if (!c.sync()) return;
      { QEps<R> b; b.n = n; b.pt = pt; b.u = u; b.q = q; b.mv1 = m1; b.mv2 = m2; c.phase(b); }
      if (!c.sync()) return;
      { QVT<R> e; e.n = n; e.pt = pt; e.u = u; e.v = v; e.w = wv; e.vt = vt; e.wt = wt; c.phase(e); }
      if (!c.sync()) return;
      { QDX<R> f; f.n = n; f.p = pv; f.pt = pt; f.d = dv; f.s = sv; f.x = x; f.r = r; f.vt = vt; f.wt = wt; f.v = v;
        f.w = wv; c.phase(f); }
      if (!c.sync()) return;
    } else {  // COCG
      cx<R>*r = V[0], *pv = V[1], *q = V[2];
      MvOut<R> mq = c.sweep_n(pv, q);
      if (!c.sync()) return;
      { CoMu<R> a; a.n = n; a.q = q; a.p = pv; a.mv = mq; c.phase(a); }
      if (!c.sync()) return;
      { CoXR<R> b; b.n = n; b.x = x; b.r = r; b.p = pv; b.q = q; c.phase(b); }
      if (!c.sync()) return;
      { CoP<R> e; e.n = n; e.r = r; e.p = pv; c.phase(e); }
      if (!c.sync()) return;
    }
  }
}

template <class R, int U, int M>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 8 ? 2 : 3) pk_solve(const PkSys<R>* __restrict__ sys, int count, long long limit,
                                                      int* fault, int withhold) {
  __shared__ cx<R> tsm[tile_smem_elems<R, U, 4>()];
  int lo = 0, hi = count - 1;  // the group of this block: largest g with sys[g].b0 <= blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (sys[mid].b0 <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const PkSys<R>& S = sys[lo];
  const int lb = (int)blockIdx.x - S.b0;
  if (lb < 0 || lb >= S.nb) return;
  if (withhold && lo == 0 && lb == 0 && S.nb > 1) return;  // test hook: never arrive
  PkCtx<R, U> c(S, lb, S.nb, limit, fault, tsm);
  pk_run_group<R, U, M>(c);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
#define PK_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));               \
      return CCG_ERR_CUDA;                                                         \
    }                                                                              \
  } while (0)

// The tuned choice for a single solve (tune_table.h); false: the kernel loop.
static bool pk_tuned(int dtype, int method, int64_t n, int* blocks) {
  for (const TuneEntry& e : kTune) {
    if (e.dtype == dtype && e.method == method && n <= e.nmax) {
      *blocks = e.pk_blocks;
      return e.persistent != 0;
    }
  }
  return false;
}

bool pk_eligible(const ccg_handle* h, int method, const ccg_operator* op) {
  if (op->kind != CCG_OPK_DENSE || !(method == M_BICGSTAB || method == M_CGNR || method == M_QMR || method == M_COCG))
    return false;
  if (h->persistent == 1) return true;
  int blocks = 0;
  return h->persistent == 2 && pk_tuned(op->dtype, method, op->n, &blocks);
}

// Resident blocks per SM of the persistent kernel (occupancy calculator,
// capped by the handle's CCG_OPT_PK_BLOCKS).
// The kernel for a precision, load width and method.
template <class R, int U> static const void* pk_kernel(int method) {
  switch (method) {
    case M_BICGSTAB: return (const void*)pk_solve<R, U, M_BICGSTAB>;
    case M_CGNR: return (const void*)pk_solve<R, U, M_CGNR>;
    case M_QMR: return (const void*)pk_solve<R, U, M_QMR>;
    case M_REFRES:
      if constexpr (sizeof(R) == 8) return (const void*)pk_solve<R, U, M_REFRES>;
      return nullptr;
    default: return (const void*)pk_solve<R, U, M_COCG>;
  }
}

// Resident blocks per SM of a persistent kernel (occupancy calculator, capped
// by the handle's CCG_OPT_PK_BLOCKS).
static int pk_blocks_per_sm(const ccg_handle* h, const void* fn, int tuned = 0) {
  int o = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, kBlock, 0) != cudaSuccess) {
    cudaGetLastError();
    o = 1;
  }
  o = std::max(1, o);
  const int want = h->pk_blocks > 0 ? h->pk_blocks : tuned;
  return want > 0 ? std::min(o, want) : o;
}

// Blocks per system: every system at least one, the rest in proportion to its
// matrix bytes (largest remainders first).
static std::vector<int> pk_groups(const std::vector<double>& work, int total) {
  const int m = (int)work.size();
  std::vector<int> nb(m, 1);
  double sum = 0.0;
  for (double w : work) sum += w;
  int left = total - m;
  if (left <= 0 || sum <= 0.0) return nb;
  std::vector<std::pair<double, int>> rem;
  int used = 0;
  for (int s = 0; s < m; ++s) {
    const double share = left * work[s] / sum;
    const int whole = (int)share;
    nb[s] += whole;
    used += whole;
    rem.push_back({share - whole, s});
  }
  std::sort(rem.begin(), rem.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
    return a.first > b.first || (a.first == b.first && a.second < b.second);
  });
  for (int k = 0; k < left - used && k < m; ++k) nb[rem[k].second] += 1;
  return nb;
}

template <class R>
int pk_solve_jobs(ccg_handle* h, int method, int count, const PkJob<R>* jobs, char* meta) {
  if (count < 1) return CCG_OK;
  cudaStream_t s = h->stream;
  // 16-byte loads of two complex64 values only when every system allows them
  // (the jobs' workspaces were laid out for the same width: PkJob::unit)
  bool wide = sizeof(R) == 4;
  for (int k = 0; k < count; ++k) wide = wide && jobs[k].op->unit == 2 && jobs[k].unit != 1;
  const void* fn = pk_kernel<R, 1>(method);
  if constexpr (sizeof(R) == 4) {
    if (wide) fn = pk_kernel<R, 2>(method);
  }
  int tuned = 0;
  if (count == 1 && h->persistent == 2) pk_tuned(jobs[0].op->dtype, method, jobs[0].op->n, &tuned);
  const int total = h->num_sms * pk_blocks_per_sm(h, fn, tuned);
  if (count > total) {
    set_error("persistent solve: more systems (" + std::to_string(count) + ") than resident blocks (" +
              std::to_string(total) + ")");
    return CCG_ERR_INVALID;
  }
  std::vector<double> work(count);
  for (int k = 0; k < count; ++k) work[k] = (double)jobs[k].op->n * (double)jobs[k].op->n;
  const std::vector<int> nb = pk_groups(work, total);

  // launch descriptors, barriers and the fault flag in a device block of the
  // arena placed after the jobs' workspaces (the caller reserved it)
  const size_t sys_bytes = align256((size_t)count * sizeof(PkSys<R>));
  const size_t bar_bytes = align256((size_t)count * sizeof(GroupBar));
  PkSys<R>* dsys = reinterpret_cast<PkSys<R>*>(meta);
  GroupBar* dbar = reinterpret_cast<GroupBar*>(meta + sys_bytes);
  int* dfault = reinterpret_cast<int*>(meta + sys_bytes + bar_bytes);
  int* dfxe = reinterpret_cast<int*>(meta + sys_bytes + bar_bytes + 256);

  std::vector<PkSys<R>> hs(count);
  int b0 = 0;
  for (int k = 0; k < count; ++k) {
    const PkJob<R>& j = jobs[k];
    const Dense<R> d(j.op, h->num_sms, j.unit);
    PkSys<R>& S = hs[k];
    std::memset(&S, 0, sizeof(S));
    S.A = d.A; S.lda = d.lda; S.n = d.n; S.unit = d.unit; S.ncb = d.ncb;
    if (d.unit != (wide ? 2 : 1)) {  // the workspace's partial sums are sized for d.unit
      set_error("persistent solve: complex64 systems of one launch must share their load width");
      return CCG_ERR_INVALID;
    }
    S.ns_c = d.tc.nsplit; S.rpr_c = d.tc.rows_per_range;
    S.ns_b = d.tb.nsplit; S.rpr_b = d.tb.rows_per_range;
    S.y = j.y; S.x = j.x;
    for (int i = 0; i < 12; ++i) S.V[i] = j.w.vec[i];
    S.P1 = j.w.P1; S.P2 = j.w.P2;
    S.st = j.w.st; S.partials = j.w.partials; S.counter = j.w.counter; S.bar = dbar + k;
    S.b0 = b0; S.nb = nb[k];
    S.method = method; S.x0_zero = j.x0_zero ? 1 : 0;
    S.nvb = phase_grid(h, d.n);
    S.r32 = j.r32; S.d32 = j.d32; S.outer = j.outer;
    S.want_true = j.want_true ? 1 : 0; S.scratch = j.w.scratch;
    S.fxC = nullptr; S.fxrow = nullptr; S.xfx = nullptr; S.xfx2 = nullptr; S.fxe = dfxe + 4 * k;
    if (sizeof(R) == 8 && h->fx_mode && j.w.xfx != nullptr && fx_prepare(h, j.op)) {
      const char* base = static_cast<const char*>(j.op->fx_a);
      S.fxC = reinterpret_cast<const int4*>(base);
      S.fxrow = reinterpret_cast<const int*>(base + (size_t)d.n * d.n * sizeof(int4) + 256);
      S.xfx = j.w.xfx;
      S.xfx2 = j.w.xfx2;
    }
    b0 += nb[k];

    if (!j.keep_state) {
      SolveState init;
      std::memset(&init, 0, sizeof(init));
      init.maxit = j.maxit;
      init.tol = j.tol;
      init.hist = j.w.hist;
      init.skip_mv = j.x0_zero ? 0 : 1;
      PK_CUDA(cudaMemcpyAsync(j.w.st, &init, sizeof(init), cudaMemcpyHostToDevice, s));
      PK_CUDA(cudaMemsetAsync(j.w.counter, 0, sizeof(unsigned int), s));
      if (j.x0_zero) PK_CUDA(cudaMemsetAsync(j.x, 0, j.op->n * sizeof(cx<R>), s));
    } else {
      // a refinement step: the state carries over; the step is not done yet
      PK_CUDA(cudaMemsetAsync(&j.w.st->poll.done, 0, sizeof(int), s));
    }
  }
  PK_CUDA(cudaMemcpyAsync(dsys, hs.data(), (size_t)count * sizeof(PkSys<R>), cudaMemcpyHostToDevice, s));
  PK_CUDA(cudaMemsetAsync(dbar, 0, bar_bytes + 256 + (size_t)count * 4 * sizeof(int), s));

  const long long limit = h->wait_limit;
  const int withhold = h->test_withhold == 1;
  void* args[] = {(void*)&dsys, (void*)&count, (void*)&limit, (void*)&dfault, (void*)&withhold};
  timing_begin(h);
  PK_CUDA(cudaLaunchCooperativeKernel(fn, dim3(b0), dim3(kBlock), args, 0, s));
  ++h->launches;
  timing_end(h, sizeof(R) == 8 ? CCG_C128 : CCG_C64, CCG_SWEEP_PERSIST, 0.0);
  int fault = 0;
  PK_CUDA(cudaMemcpyAsync(&fault, dfault, sizeof(int), cudaMemcpyDeviceToHost, s));
  for (int k = 0; k < count; ++k)
    PK_CUDA(cudaMemcpyAsync(jobs[k].fin, jobs[k].w.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  PK_CUDA(cudaStreamSynchronize(s));
  if (h->timing) {
    // the launch counts as the sweeps it ran, each of one matrix's bytes
    int64_t sweeps = 0;
    double bytes = 0.0;
    for (int k = 0; k < count; ++k) {
      sweeps += jobs[k].fin->sweeps;
      bytes += (double)jobs[k].fin->sweeps * (double)jobs[k].op->n * (double)jobs[k].op->n * sizeof(cx<R>);
    }
    timing_set_units(h, sweeps, bytes);
  }
  if (fault) {
    set_error("persistent solve: a group barrier gave up waiting (CCG_ERR_TIMEOUT)");
    return CCG_ERR_TIMEOUT;
  }
  if (method != M_REFRES) {
    for (int k = 0; k < count; ++k) {
      if (!jobs[k].fin->poll.done) {
        set_error("persistent solve did not record its end");
        return CCG_ERR_CUDA;
      }
    }
  }
  return CCG_OK;
}

// ---------------------------------------------------------------------------
// Many systems in one launch (ccg_solve_multi, ccg_solve_multi_refined).
// ---------------------------------------------------------------------------
// Load width shared by a launch's complex64 systems: pairs only if all allow.
static int common_unit(int count, const ccg_operator* const* ops) {
  for (int k = 0; k < count; ++k)
    if (ops[k]->unit != 2) return 1;
  return 2;
}

template <class R>
static std::vector<Ws<R>> carve_all(ccg_handle* h, int count, const ccg_operator* const* ops, int maxit, int unit,
                                    char* base, size_t* used) {
  std::vector<Ws<R>> ws;
  size_t off = 0;
  for (int k = 0; k < count; ++k) {
    const Dense<R> d(ops[k], h->num_sms, unit);
    ws.push_back(ws_carve<R>(base + off, ops[k]->n, d, maxit));
    off += ws_bytes<R>(ops[k]->n, d, maxit);
  }
  *used = off;
  return ws;
}

template <class R>
static size_t bytes_all(ccg_handle* h, int count, const ccg_operator* const* ops, int maxit, int unit) {
  size_t b = 0;
  for (int k = 0; k < count; ++k) {
    const Dense<R> d(ops[k], h->num_sms, unit);
    b += ws_bytes<R>(ops[k]->n, d, maxit);
  }
  return b;
}

template <class R>
static int multi_t(ccg_handle* h, int method, int count, const ccg_operator* const* ops, const void* const* y,
                   void* const* x, const double* tol, int maxit, int32_t* iters, int32_t* status, double* relres) {
  const int unit = sizeof(R) == 4 ? common_unit(count, ops) : 1;
  const size_t wb = bytes_all<R>(h, count, ops, maxit, unit);
  int rc = arena_reserve(h, wb + pk_meta_bytes(count, sizeof(R) == 8 ? CCG_C128 : CCG_C64));
  if (rc != CCG_OK) return rc;
  size_t used = 0;
  std::vector<Ws<R>> ws = carve_all<R>(h, count, ops, maxit, unit, h->arena, &used);
  std::vector<SolveState> fin(count);
  std::vector<PkJob<R>> jobs(count);
  for (int k = 0; k < count; ++k) {
    PkJob<R>& j = jobs[k];
    j.op = ops[k]; j.w = ws[k]; j.y = static_cast<const cx<R>*>(y[k]); j.x = static_cast<cx<R>*>(x[k]);
    j.tol = tol[k]; j.maxit = maxit; j.x0_zero = false; j.fin = &fin[k]; j.want_true = true; j.unit = unit;
  }
  if ((rc = pk_solve_jobs<R>(h, method, count, jobs.data(), h->arena + wb)) != CCG_OK) return rc;
  cudaStream_t s = h->stream;
  std::vector<double> rr(count, 0.0);
  for (int k = 0; k < count; ++k) {
    PK_CUDA(cudaMemcpyAsync(&rr[k], ws[k].scratch, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (fin[k].zero_rhs) PK_CUDA(cudaMemsetAsync(x[k], 0, ops[k]->n * sizeof(cx<R>), s));
  }
  PK_CUDA(cudaStreamSynchronize(s));
  int worst = CCG_OK;
  for (int k = 0; k < count; ++k) {
    const int st = fin[k].poll.status;
    if (iters) iters[k] = fin[k].poll.k;
    if (status) status[k] = st;
    if (relres) relres[k] = fin[k].poll.ynorm > 0 ? std::sqrt(rr[k]) / fin[k].poll.ynorm : 0.0;
    if (st < 0) worst = std::min(worst, st);
    else if (worst >= 0) worst = std::max(worst, st);
  }
  return worst;
}

int solve_multi(ccg_handle* h, int method, int count, const ccg_operator* const* ops, const void* const* y,
                void* const* x, const double* tol, int maxit, int32_t* iters, int32_t* status, double* relres) {
  if (ops[0]->dtype == CCG_C128) return multi_t<double>(h, method, count, ops, y, x, tol, maxit, iters, status, relres);
  return multi_t<float>(h, method, count, ops, y, x, tol, maxit, iters, status, relres);
}

int solve_multi_refined(ccg_handle* h, int method, int count, const ccg_operator* const* ops,
                        const ccg_operator* const* ops_in, const void* const* y, void* const* x, const double* tol,
                        int max_outer, double inner_tol, int inner_maxit, int32_t* outer_out, int32_t* inner_out,
                        int32_t* status, double* relres) {
  const int unit = common_unit(count, ops_in);
  const size_t b64 = bytes_all<double>(h, count, ops, max_outer, 1);
  const size_t b32 = bytes_all<float>(h, count, ops_in, inner_maxit, unit);
  int rc = arena_reserve(h, b64 + b32 + pk_meta_bytes(count, CCG_C128));
  if (rc != CCG_OK) return rc;
  size_t used = 0;
  std::vector<Ws<double>> w64 = carve_all<double>(h, count, ops, max_outer, 1, h->arena, &used);
  std::vector<Ws<float>> w32 = carve_all<float>(h, count, ops_in, inner_maxit, unit, h->arena + b64, &used);
  char* meta = h->arena + b64 + b32;
  std::vector<SolveState> f64(count), f32(count);
  std::vector<int> outer(count, 0), inner(count, 0), st(count, CCG_NOT_CONVERGED), active;
  for (int k = 0; k < count; ++k) active.push_back(k);
  cudaStream_t s = h->stream;
  while (!active.empty()) {
    // x += d (after the first step), r = y - A x and the stopping test, for
    // every system still refining, in one launch
    std::vector<PkJob<double>> jr;
    for (int k : active) {
      PkJob<double> j;
      j.op = ops[k]; j.w = w64[k]; j.y = static_cast<const double2*>(y[k]); j.x = static_cast<double2*>(x[k]);
      j.tol = tol[k]; j.maxit = max_outer; j.x0_zero = false; j.fin = &f64[k];
      j.keep_state = outer[k] > 0; j.r32 = w32[k].ystage; j.d32 = w32[k].xstage; j.outer = outer[k];
      jr.push_back(j);
    }
    if ((rc = pk_solve_jobs<double>(h, M_REFRES, (int)jr.size(), jr.data(), meta)) != CCG_OK) return rc;
    std::vector<int> next;
    for (int k : active) {
      if (f64[k].poll.done) st[k] = f64[k].poll.status;
      else next.push_back(k);
    }
    active.swap(next);
    if (active.empty()) break;
    // the corrections A d = r in complex64, all in one launch
    std::vector<PkJob<float>> ji;
    for (int k : active) {
      PkJob<float> j;
      j.op = ops_in[k]; j.w = w32[k]; j.y = w32[k].ystage; j.x = w32[k].xstage; j.tol = inner_tol;
      j.maxit = inner_maxit; j.x0_zero = true; j.fin = &f32[k]; j.unit = unit;
      ji.push_back(j);
    }
    if ((rc = pk_solve_jobs<float>(h, method, (int)ji.size(), ji.data(), meta)) != CCG_OK) return rc;
    next.clear();
    for (int k : active) {
      inner[k] += f32[k].poll.k;
      if (f32[k].poll.status == ST_NONFINITE) { st[k] = CCG_ERR_NONFINITE; continue; }
      if (f32[k].poll.status == ST_BREAKDOWN && f32[k].poll.k == 0) { st[k] = CCG_BREAKDOWN; continue; }
      outer[k] += 1;
      next.push_back(k);
    }
    active.swap(next);
  }
  for (int k = 0; k < count; ++k)
    if (f64[k].zero_rhs) PK_CUDA(cudaMemsetAsync(x[k], 0, ops[k]->n * sizeof(double2), s));
  PK_CUDA(cudaStreamSynchronize(s));
  int worst = CCG_OK;
  for (int k = 0; k < count; ++k) {
    if (outer_out) outer_out[k] = f64[k].poll.k;
    if (inner_out) inner_out[k] = inner[k];
    if (status) status[k] = st[k];
    if (relres) relres[k] = f64[k].poll.relres;
    if (st[k] < 0) worst = std::min(worst, st[k]);
    else if (worst >= 0) worst = std::max(worst, st[k]);
  }
  return worst;
}

int pk_capacity(ccg_handle* h, int method, int dtype) {
  const void* fn = dtype == CCG_C128 ? pk_kernel<double, 1>(method) : pk_kernel<float, 1>(method);
  return fn ? h->num_sms * pk_blocks_per_sm(h, fn) : 0;
}

size_t pk_meta_bytes(int count, int dtype) {
  const size_t sys = dtype == CCG_C128 ? sizeof(PkSys<double>) : sizeof(PkSys<float>);
  return align256((size_t)count * sys) + align256((size_t)count * sizeof(GroupBar)) + 256 +
         align256((size_t)count * 4 * sizeof(int));
}

template int pk_solve_jobs<double>(ccg_handle*, int, int, const PkJob<double>*, char*);
template int pk_solve_jobs<float>(ccg_handle*, int, int, const PkJob<float>*, char*);

}  // namespace ccg
