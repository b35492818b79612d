// Launch geometry of the dense sweeps and the layout of a solve's workspace
// in the handle's arena (vectors, partial sums, reduction slots, device
// solve state, residual history, GMRES basis), shared by the multi-kernel
// solve loop (solve.cu) and the persistent solve (persist.cu).
#pragma once

#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "reduce.cuh"
#include "gemv.cuh"
#include "fx.cuh"
#include "internal.h"

namespace ccg {

// GMRES(m) workspace: Hessenberg matrix, rotations and the passes' partials.
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

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Warps per matrix row in the row sweep (gemv_n_rows), and in the
// fixed-point complex128 row sweep (gemv_fx_rows).
constexpr int kRowSplit = 4;
constexpr int kFxSplit = 2;

// Launch geometry of the dense sweeps for one operator.
// Resident blocks per SM of the column-tiled sweep (A^H x alone, or A x1 with
// A^H x2), from the occupancy calculator; for complex128 A^H x that of the
// integer-pipe sweep (the default; the FP64-pipe fallback runs the same
// tiles).
template <class R> static int tile_occupancy(int unit, bool both) {
  static int cache[2][2] = {{0, 0}, {0, 0}};
  int& c = cache[unit == 2 ? 1 : 0][both ? 1 : 0];
  if (c == 0) {
    const void* fn = nullptr;
    if constexpr (sizeof(R) == 4) {
      if (unit == 2) fn = both ? (const void*)gemv_tile<R, 2, 4, true, true> : (const void*)gemv_tile_h<R, 2, 4>;
      else fn = both ? (const void*)gemv_tile<R, 1, 4, true, true> : (const void*)gemv_tile_h<R, 1, 4>;
    } else {
      fn = both ? (const void*)gemv_tile<R, 1, 4, true, true> : (const void*)gemv_fx_tile_h;
    }
    // the integer A^H sweep stages its rows in dynamic shared memory
    const size_t dyn = (sizeof(R) == 8 && !both) ? kFxTileSmem : 0;
    if (dyn > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kBlock, dyn) != cudaSuccess) {
      cudaGetLastError();
      occ = 2;
    }
    c = std::max(1, occ);
  }
  return c;
}

// Row ranges of a column-tiled sweep: the number of ranges ns (1 .. 32, at
// least 8 rows each) whose ncb x ns tiles finish soonest on `slots`
// resident blocks -- ceil(tiles / slots) waves of tiles of 1/tiles of the
// work each -- the fewest ranges among equals.  (Filling the slots once with
// a few tiles to spare left a second wave of those few.)
struct TileSplit {
  int nsplit;
  int64_t rows_per_range;
};
static TileSplit tile_split(int64_t n, int ncb, int64_t slots) {
  const int64_t cap = std::max<int64_t>(1, std::min<int64_t>(32, (n + kWarps - 1) / kWarps));
  slots = std::max<int64_t>(1, slots);
  int64_t ns = 1;
  double best = 1e300;
  for (int64_t k = 1; k <= cap; ++k) {
    const int64_t tiles = (int64_t)ncb * k;
    const double t = (double)((tiles + slots - 1) / slots) / (double)tiles;
    if (t < best * (1.0 - 1e-12)) {
      best = t;
      ns = k;
    }
  }
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
  int grid_fx;              // gemv_fx_rows blocks
  int ncb;                  // gemv_tile column chunks
  TileSplit tc, tb;         // row ranges for A^H x, and for A x1 with A^H x2
  static constexpr int E = 4;

  // unit_override 1: single-element loads even where 16-byte pairs are
  // allowed (a persistent launch whose systems differ in that)
  Dense(const ccg_operator* op, int num_sms, int unit_override = 0) {
    A = static_cast<const cx<R>*>(op->A);
    lda = op->lda;
    n = op->n;
    unit = unit_override > 0 ? unit_override : op->unit;
    grid_rows = (int)std::min<int64_t>((n + kWarps / kRowSplit - 1) / (kWarps / kRowSplit), 1 << 30);
    grid_fx = (int)std::min<int64_t>((n + kWarps / kFxSplit - 1) / (kWarps / kFxSplit), 1 << 30);
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

// Grid of the fused update kernels ("phases"): one element per thread up to
// about 2.7 blocks per SM (on large systems fewer, longer-running blocks
// leave less to the cross-block reduction: on the 412k-unknown dipole system
// 405 blocks beat 1216 by 7%; n = 8192 keeps 32); the handle's floor on
// elements per thread applies.
static inline int phase_grid(const ccg_handle* h, int64_t n) {
  const int64_t per_block = (int64_t)kBlock * h->phase_elems;
  int g = (int)std::min<int64_t>((n + per_block - 1) / per_block, (int64_t)h->num_sms * 8 / 3);
  return std::max(1, std::min(g, kMaxRedBlocks));
}

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
  int4* xfx;        // complex128: the digits of a sweep's vector (fx.cuh)
  int* xmeta;       // and its exponent and non-finite flag
  int4* xfx2;       // the row-scaled vector of an A^H x sweep, and its exponent
  int* xmeta2;
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
  if (sizeof(R) == 8) b += 2 * (align256(n * sizeof(int4)) + align256(4 * sizeof(int)));
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
  w.xfx = w.xfx2 = nullptr;
  w.xmeta = w.xmeta2 = nullptr;
  if (sizeof(R) == 8) {
    w.xfx = reinterpret_cast<int4*>(take(n * sizeof(int4)));
    w.xmeta = reinterpret_cast<int*>(take(4 * sizeof(int)));
    w.xfx2 = reinterpret_cast<int4*>(take(n * sizeof(int4)));
    w.xmeta2 = reinterpret_cast<int*>(take(4 * sizeof(int)));
  }
  return w;
}


// ---------------------------------------------------------------------------
// Persistent solves (persist.cu).
// ---------------------------------------------------------------------------
struct GroupBar {
  unsigned count;       // arrivals since the launch began (G per barrier)
  unsigned pad[31];     // one 128-byte line per group
};

// One system of a persistent launch: its operator geometry, workspace and
// block range [b0, b0 + nb).
template <class R> struct PkSys {
  const cx<R>* A;
  int64_t lda, n;
  int unit, ncb;
  int ns_c, ns_b;            // row ranges of the A^H x sweep and of the fused sweep
  int64_t rpr_c, rpr_b;      // rows per range
  const cx<R>* y;
  cx<R>* x;
  cx<R>* V[12];
  cx<R>* P1;
  cx<R>* P2;
  SolveState* st;
  double* partials;
  unsigned int* counter;
  GroupBar* bar;
  int b0, nb;
  int nvb;                   // virtual blocks of a vector phase (the kernel loop's phase grid)
  int method, x0_zero;
  // complex128 fixed-point sweep (fx.cuh): the operator's digits and row
  // exponents (null: the FP64 pipe), the vector's digits, and the group's
  // exponent words (two alternating slots)
  const int4* fxC;
  const int* fxrow;
  int4* xfx;
  int4* xfx2;                // the row-scaled vector of an A^H x sweep
  int* fxe;
  // refinement step (M_REFRES): the inner solve's right-hand side and
  // correction (complex64), the outer step's index; and whether the group
  // forms the final true residual ||y - A x||^2 into its scratch
  float2* r32;
  float2* d32;
  int outer;
  int want_true;
  double* scratch;
};

// A solve to run in a persistent launch: operator, workspace, right-hand
// side, start vector (solution out), tolerance and cap; *fin receives the
// final device state.
template <class R> struct PkJob {
  const ccg_operator* op;
  Ws<R> w;
  const cx<R>* y;
  cx<R>* x;
  double tol;
  int maxit;
  bool x0_zero;
  SolveState* fin;
  int unit = 0;              // the launch's load width, when it overrides the operator's
  bool keep_state = false;   // a later refinement step: the device state carries over
  bool want_true = false;    // form ||y - A x||^2 after the iteration (into w.scratch[0])
  float2* r32 = nullptr;     // refinement step: inner right-hand side and correction
  float2* d32 = nullptr;
  int outer = 0;
};

// The refinement step as a persistent "method": x += d (after the first
// step), r = y - A x, the stopping test, r32 = round(r), d32 = 0.
constexpr int M_REFRES = 100;

// Whether a solve runs persistently (the handle's option, a dense operator,
// BiCGSTAB, CGNR, QMR or COCG).
bool pk_eligible(const ccg_handle* h, int method, const ccg_operator* op);
// Device bytes a launch of `count` systems needs beside their workspaces.
size_t pk_meta_bytes(int count, int dtype);
// Run the jobs in one cooperative launch on the handle's stream, using `meta`
// (pk_meta_bytes) for the launch's descriptors; returns with the stream idle.
template <class R> int pk_solve_jobs(ccg_handle* h, int method, int count, const PkJob<R>* jobs, char* meta);

}  // namespace ccg
