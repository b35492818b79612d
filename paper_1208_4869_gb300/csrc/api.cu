// C ABI of libccg (include/ccg.h): handles, operators, argument checks,
// workspace, timing, and dispatch to the solver and operator code.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace ccg {

static thread_local std::string g_error = "";

void set_error(const std::string& msg) { g_error = msg; }

#define API_CUDA(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                   \
      return CCG_ERR_CUDA;                                                             \
    }                                                                                  \
  } while (0)

int arena_reserve(ccg_handle* h, size_t bytes) {
  if (bytes <= h->arena_bytes) return CCG_OK;
  if (h->arena) {
    API_CUDA(cudaStreamSynchronize(h->stream));
    API_CUDA(cudaFree(h->arena));
    h->arena = nullptr;
    h->arena_bytes = 0;
  }
  const size_t want = bytes + bytes / 8;  // headroom against small growth steps
  if (cudaMalloc(&h->arena, want) != cudaSuccess) {
    cudaGetLastError();
    h->arena = nullptr;
    set_error("workspace allocation of " + std::to_string(want) + " bytes failed");
    return CCG_ERR_NOMEM;
  }
  h->arena_bytes = want;
  return CCG_OK;
}

void timing_begin(ccg_handle* h) {
  if (!h->timing) return;
  if (h->tev_used + 2 > h->tev.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      h->tev.push_back(e);
      h->tev_kind.push_back(0);
      h->tev_units.push_back(1);
      h->tev_bytes.push_back(0.0);
    }
  }
  cudaEventRecord(h->tev[h->tev_used], h->stream);
}

void timing_end(ccg_handle* h, int dtype, int kind, double bytes) {
  if (!h->timing) return;
  const int slot = dtype * CCG_SWEEP_KINDS + kind;
  cudaEventRecord(h->tev[h->tev_used + 1], h->stream);
  h->tev_kind[h->tev_used] = slot;
  h->tev_units[h->tev_used] = 1;
  h->tev_bytes[h->tev_used] = bytes;
  h->tev_used += 2;
  h->bytes_per_sweep[slot] = bytes;
}

void timing_set_units(ccg_handle* h, int64_t units, double bytes) {
  if (!h->timing || h->tev_used < 2) return;
  h->tev_units[h->tev_used - 2] = units;
  h->tev_bytes[h->tev_used - 2] = bytes;
}

int* timing_rec(ccg_handle* h) {
  if (!h->timing || !h->skip_rec || h->tev_used / 2 >= h->skip_cap) return nullptr;
  return h->skip_rec + h->tev_used / 2;
}

// Sum the recorded sweep durations (the stream must be idle) and recycle the
// events.  Sweeps that found the solve already stopped (enqueued ahead of
// the convergence test) returned at once and are left out.
void timing_collect(ccg_handle* h) {
  const size_t pairs = h->tev_used / 2;
  std::vector<int> skipped(pairs, 0);
  if (h->skip_rec && pairs > 0) {
    const size_t m = std::min(pairs, h->skip_cap);
    if (cudaMemcpy(skipped.data(), h->skip_rec, m * sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
      cudaMemsetAsync(h->skip_rec, 0, m * sizeof(int), h->stream);
  }
  for (size_t i = 0; i + 1 < h->tev_used; i += 2) {
    float ms = 0.f;
    if (skipped[i / 2] || h->tev_units[i] <= 0) continue;
    if (cudaEventElapsedTime(&ms, h->tev[i], h->tev[i + 1]) == cudaSuccess) {
      h->timed_ms[h->tev_kind[i]] += ms;
      h->timed_sweeps[h->tev_kind[i]] += h->tev_units[i];
      h->timed_bytes[h->tev_kind[i]] += h->tev_bytes[i];   // a pair's bytes in total
    }
  }
  cudaGetLastError();
  h->tev_used = 0;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace ccg

using namespace ccg;

extern "C" {

int ccg_abi_version(void) { return CCG_ABI_VERSION; }

const char* ccg_last_error(void) { return g_error.c_str(); }

const char* ccg_status_string(int status) {
  switch (status) {
    case CCG_OK: return "converged";
    case CCG_NOT_CONVERGED: return "iteration cap reached";
    case CCG_BREAKDOWN: return "breakdown";
    case CCG_ERR_INVALID: return "invalid argument";
    case CCG_ERR_NOMEM: return "out of device memory";
    case CCG_ERR_CUDA: return "CUDA error";
    case CCG_ERR_NONFINITE: return "non-finite value";
    case CCG_ERR_TIMEOUT: return "device wait timed out";
    case CCG_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

ccg_status ccg_create(ccg_handle** out, void* stream) {
  if (!out) { set_error("ccg_create: NULL output"); return CCG_ERR_INVALID; }
  *out = nullptr;
  int dev = 0, count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    set_error("ccg_create: no CUDA device");
    return CCG_ERR_CUDA;
  }
  API_CUDA(cudaGetDevice(&dev));
  ccg_handle* h = new (std::nothrow) ccg_handle();
  if (!h) { set_error("ccg_create: host allocation failed"); return CCG_ERR_NOMEM; }
  h->stream = static_cast<cudaStream_t>(stream);
  h->device = dev;
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (h->num_sms <= 0) h->num_sms = 1;
  if (const char* e = std::getenv("CCG_PHASE_MIN_ELEMS")) {  // tuning override of the fused-kernel grid
    const int v = std::atoi(e);
    if (v >= 1 && v <= 64) h->phase_elems = v;
  }
  if (cudaHostAlloc(&h->pinned, 2 * sizeof(Poll), cudaHostAllocDefault) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->poll_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->poll_ev[1], cudaEventDisableTiming) != cudaSuccess) {
    set_error(std::string("ccg_create: ") + cudaGetErrorString(cudaGetLastError()));
    ccg_destroy(h);
    return CCG_ERR_CUDA;
  }
  std::memset(h->pinned, 0, 2 * sizeof(Poll));
  *out = h;
  return CCG_OK;
}

ccg_status ccg_destroy(ccg_handle* h) {
  if (!h) return CCG_OK;
  cudaStreamSynchronize(h->stream);
  if (h->arena) cudaFree(h->arena);
  if (h->tc_buf) cudaFree(h->tc_buf);
  if (h->oz_buf) cudaFree(h->oz_buf);
  if (h->pinned) cudaFreeHost(h->pinned);
  if (h->skip_rec) cudaFree(h->skip_rec);
  for (int i = 0; i < 2; ++i)
    if (h->poll_ev[i]) cudaEventDestroy(h->poll_ev[i]);
  for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
  cudaGetLastError();
  delete h;
  return CCG_OK;
}

ccg_status ccg_set_stream(ccg_handle* h, void* stream) {
  if (!h) { set_error("ccg_set_stream: NULL handle"); return CCG_ERR_INVALID; }
  API_CUDA(cudaStreamSynchronize(h->stream));
  h->stream = static_cast<cudaStream_t>(stream);
  return CCG_OK;
}

ccg_status ccg_op_dense(ccg_handle* h, ccg_dtype dtype, int64_t n, const void* A, int64_t lda, int flags,
                        ccg_operator** op) {
  if (!op) { set_error("ccg_op_dense: NULL output"); return CCG_ERR_INVALID; }
  *op = nullptr;
  if (!h || !A) { set_error("ccg_op_dense: NULL handle or matrix"); return CCG_ERR_INVALID; }
  if (dtype != CCG_C64 && dtype != CCG_C128) { set_error("ccg_op_dense: bad dtype"); return CCG_ERR_INVALID; }
  if (n < 1 || lda < n) { set_error("ccg_op_dense: need n >= 1 and lda >= n"); return CCG_ERR_INVALID; }
  if (n > (int64_t(1) << 31)) { set_error("ccg_op_dense: n too large"); return CCG_ERR_INVALID; }
  const size_t esz = dtype == CCG_C128 ? 16 : 8;
  if (!aligned(A, esz)) { set_error("ccg_op_dense: matrix not aligned to its element size"); return CCG_ERR_INVALID; }
  if (flags & ~CCG_OP_SYMMETRIC) { set_error("ccg_op_dense: unknown flags"); return CCG_ERR_INVALID; }
  ccg_operator* o = new (std::nothrow) ccg_operator();
  if (!o) { set_error("ccg_op_dense: host allocation failed"); return CCG_ERR_NOMEM; }
  o->kind = CCG_OPK_DENSE;
  o->dtype = dtype;
  o->n = n;
  o->flags = flags;
  o->A = A;
  o->lda = lda;
  o->unit = 1;
  if (dtype == CCG_C64 && (n % 2 == 0) && (lda % 2 == 0) && aligned(A, 16)) o->unit = 2;
  *op = o;
  return CCG_OK;
}

ccg_status ccg_op_dipole(ccg_handle* h, ccg_dtype dtype, int nx, int ny, int nz, const uint8_t* occ, double kd,
                         double m_re, double m_im, ccg_operator** op) {
  if (!op) { set_error("ccg_op_dipole: NULL output"); return CCG_ERR_INVALID; }
  *op = nullptr;
  if (!h || !occ) { set_error("ccg_op_dipole: NULL handle or occupancy"); return CCG_ERR_INVALID; }
  if (dtype != CCG_C64 && dtype != CCG_C128) { set_error("ccg_op_dipole: bad dtype"); return CCG_ERR_INVALID; }
  if (nx < 1 || ny < 1 || nz < 1 || !(kd >= 0.0) || !std::isfinite(m_re) || !std::isfinite(m_im)) {
    set_error("ccg_op_dipole: need nx, ny, nz >= 1, kd >= 0 and a finite refractive index");
    return CCG_ERR_INVALID;
  }
  // Clausius-Mossotti polarizability (unit lattice spacing)
  const std::complex<double> m(m_re, m_im), m2 = m * m;
  const std::complex<double> alpha = (3.0 / (4.0 * M_PI)) * (m2 - 1.0) / (m2 + 2.0);
  if (std::abs(alpha) == 0.0) { set_error("ccg_op_dipole: m^2 = 1 gives zero polarizability"); return CCG_ERR_INVALID; }
  int64_t count = 0;
  for (int64_t c = 0; c < (int64_t)nx * ny * nz; ++c) count += occ[c] != 0;
  if (count == 0) { set_error("ccg_op_dipole: no occupied site"); return CCG_ERR_INVALID; }
  ccg_operator* o = new (std::nothrow) ccg_operator();
  if (!o) { set_error("ccg_op_dipole: host allocation failed"); return CCG_ERR_NOMEM; }
  o->kind = CCG_OPK_DIPOLE;
  o->dtype = dtype;
  o->flags = CCG_OP_SYMMETRIC;
  o->dip.nx = nx;
  o->dip.ny = ny;
  o->dip.nz = nz;
  o->dip.kd = kd;
  const std::complex<double> ainv = 1.0 / alpha;
  o->dip.alpha_inv[0] = ainv.real();
  o->dip.alpha_inv[1] = ainv.imag();
  const int rc = dipole_create(o, occ, h->stream);
  if (rc != CCG_OK) {
    dipole_free(o);
    delete o;
    return static_cast<ccg_status>(rc);
  }
  *op = o;
  return CCG_OK;
}

ccg_status ccg_op_callback(ccg_handle* h, ccg_dtype dtype, int64_t n, ccg_matvec_fn matvec, ccg_matvec_fn cmatvec,
                           void* ctx, int flags, ccg_operator** op) {
  if (!op) { set_error("ccg_op_callback: NULL output"); return CCG_ERR_INVALID; }
  *op = nullptr;
  if (!h || !matvec) { set_error("ccg_op_callback: NULL handle or matvec"); return CCG_ERR_INVALID; }
  if (dtype != CCG_C64 && dtype != CCG_C128) { set_error("ccg_op_callback: bad dtype"); return CCG_ERR_INVALID; }
  if (n < 1 || n > (int64_t(1) << 31)) { set_error("ccg_op_callback: need 1 <= n <= 2^31"); return CCG_ERR_INVALID; }
  if (flags & ~CCG_OP_SYMMETRIC) { set_error("ccg_op_callback: unknown flags"); return CCG_ERR_INVALID; }
  ccg_operator* o = new (std::nothrow) ccg_operator();
  if (!o) { set_error("ccg_op_callback: host allocation failed"); return CCG_ERR_NOMEM; }
  o->kind = CCG_OPK_CALLBACK;
  o->dtype = dtype;
  o->n = n;
  o->flags = flags;
  o->unit = 1;
  o->cb_matvec = matvec;
  o->cb_cmatvec = cmatvec;
  o->cb_ctx = ctx;
  *op = o;
  return CCG_OK;
}

// Methods whose iterations apply A^H.
static bool needs_ah(int method) {
  return method == CCG_CGNR || method == CCG_QMR || method == CCG_BICG || method == CCG_CGNE;
}

int64_t ccg_dipole_sites(const ccg_operator* op) { return (op && op->kind == CCG_OPK_DIPOLE) ? op->dip.nsites : 0; }

ccg_status ccg_op_destroy(ccg_operator* op) {
  if (op && op->kind == CCG_OPK_DIPOLE) {
    cudaDeviceSynchronize();
    dipole_free(op);
  }
  if (op && op->tc_ready) tc_free(op);  // stream-ordered after the operator's last use
  if (op && op->oz_a) oz_free(op);
  if (op && op->fx_a) fx_free(op);
  delete op;
  return CCG_OK;
}

int64_t ccg_op_size(const ccg_operator* op) { return op ? op->n : 0; }

ccg_status ccg_matvec(ccg_handle* h, const ccg_operator* op, int trans, const void* x, void* y) {
  if (!h || !op || !x || !y) { set_error("ccg_matvec: NULL argument"); return CCG_ERR_INVALID; }
  if (trans != 0 && trans != 1) { set_error("ccg_matvec: trans must be 0 or 1"); return CCG_ERR_INVALID; }
  const size_t esz = op->dtype == CCG_C128 ? 16 : 8;
  if (!aligned(x, op->unit * esz) || !aligned(y, esz)) { set_error("ccg_matvec: misaligned vector"); return CCG_ERR_INVALID; }
  if (trans && op->kind == CCG_OPK_CALLBACK && !op->cb_cmatvec) {
    set_error("ccg_matvec: the callback operator has no cmatvec");
    return CCG_ERR_UNSUPPORTED;
  }
  return static_cast<ccg_status>(matvec_dense(h, op, trans, x, y));
}

ccg_status ccg_dot(ccg_handle* h, ccg_dtype dtype, int64_t n, const void* u, const void* v, int conj, double* out2) {
  if (!h || !u || !v || !out2) { set_error("ccg_dot: NULL argument"); return CCG_ERR_INVALID; }
  if (n < 0 || (dtype != CCG_C64 && dtype != CCG_C128)) { set_error("ccg_dot: bad size or dtype"); return CCG_ERR_INVALID; }
  if (n == 0) { out2[0] = out2[1] = 0.0; return CCG_OK; }
  return static_cast<ccg_status>(dot_device(h, dtype, n, u, v, conj ? 1 : 0, out2));
}

ccg_status ccg_solve(ccg_handle* h, ccg_method method, const ccg_operator* op, const void* y, void* x, double tol,
                     int maxit, double* res_hist, ccg_info* info) {
  if (!h || !op || !y || !x) { set_error("ccg_solve: NULL argument"); return CCG_ERR_INVALID; }
  if (method < CCG_BICGSTAB || method > CCG_BICGSTABL) { set_error("ccg_solve: unknown method"); return CCG_ERR_INVALID; }
  if (maxit < 0 || !(tol >= 0.0)) { set_error("ccg_solve: need maxit >= 0 and tol >= 0"); return CCG_ERR_INVALID; }
  if ((method == CCG_COCG || method == CCG_COCR) && !(op->flags & CCG_OP_SYMMETRIC)) {
    set_error("ccg_solve: COCG and COCR need an operator flagged CCG_OP_SYMMETRIC");
    return CCG_ERR_INVALID;
  }
  const size_t esz = op->dtype == CCG_C128 ? 16 : 8;
  if (!aligned(y, esz) || !aligned(x, op->unit * esz)) { set_error("ccg_solve: misaligned vector"); return CCG_ERR_INVALID; }
  if (needs_ah(method) && op->kind == CCG_OPK_CALLBACK && !op->cb_cmatvec) {
    set_error("ccg_solve: this method needs A^H and the callback operator has no cmatvec");
    return CCG_ERR_UNSUPPORTED;
  }
  return static_cast<ccg_status>(solve_dense(h, method, op, y, x, tol, maxit, res_hist, info));
}

ccg_status ccg_solve_refined(ccg_handle* h, ccg_method method, const ccg_operator* op, const ccg_operator* op_in,
                             const void* y, void* x, double tol, int max_outer, double inner_tol, int inner_maxit,
                             double* res_hist, int* inner_iters, ccg_info* info) {
  if (!h || !op || !op_in || !y || !x) { set_error("ccg_solve_refined: NULL argument"); return CCG_ERR_INVALID; }
  if (method < CCG_BICGSTAB || method > CCG_BICGSTABL) { set_error("ccg_solve_refined: unknown method"); return CCG_ERR_INVALID; }
  if (op->dtype != CCG_C128 || op_in->dtype != CCG_C64 || op->n != op_in->n) {
    set_error("ccg_solve_refined: need a complex128 operator and a complex64 operator of the same size");
    return CCG_ERR_INVALID;
  }
  if (!(tol >= 0.0) || max_outer < 0 || !(inner_tol > 0.0) || inner_maxit < 1) {
    set_error("ccg_solve_refined: need tol >= 0, max_outer >= 0, inner_tol > 0, inner_maxit >= 1");
    return CCG_ERR_INVALID;
  }
  if ((method == CCG_COCG || method == CCG_COCR) && !(op_in->flags & CCG_OP_SYMMETRIC)) {
    set_error("ccg_solve_refined: COCG and COCR need an inner operator flagged CCG_OP_SYMMETRIC");
    return CCG_ERR_INVALID;
  }
  if (!aligned(y, 16) || !aligned(x, 16)) { set_error("ccg_solve_refined: misaligned vector"); return CCG_ERR_INVALID; }
  if (needs_ah(method) && op_in->kind == CCG_OPK_CALLBACK && !op_in->cb_cmatvec) {
    set_error("ccg_solve_refined: this method needs A^H and the inner callback operator has no cmatvec");
    return CCG_ERR_UNSUPPORTED;
  }
  return static_cast<ccg_status>(
      solve_refined(h, method, op, op_in, y, x, tol, max_outer, inner_tol, inner_maxit, res_hist, inner_iters, info));
}

static int check_block(const ccg_operator* op, int64_t k, const void* Y, int64_t ldy, const void* X, int64_t ldx,
                       const char* who) {
  if (!op || !Y || !X) { set_error(std::string(who) + ": NULL argument"); return CCG_ERR_INVALID; }
  if (op->kind != CCG_OPK_DENSE) { set_error(std::string(who) + ": needs a dense operator"); return CCG_ERR_UNSUPPORTED; }
  if (k < 1 || k > 256 || ldy < op->n || ldx < op->n) {
    set_error(std::string(who) + ": need 1 <= nrhs <= 256 and leading dimensions >= n");
    return CCG_ERR_INVALID;
  }
  const size_t esz = op->dtype == CCG_C128 ? 16 : 8;
  if (!aligned(Y, esz) || !aligned(X, esz)) { set_error(std::string(who) + ": misaligned block"); return CCG_ERR_INVALID; }
  return CCG_OK;
}

ccg_status ccg_solve_batched(ccg_handle* h, ccg_method method, const ccg_operator* op, int64_t nrhs, const void* Y,
                             int64_t ldy, void* X, int64_t ldx, double tol, int maxit, int32_t* iters,
                             int32_t* status, double* relres) {
  if (!h) { set_error("ccg_solve_batched: NULL handle"); return CCG_ERR_INVALID; }
  if (method != CCG_BICGSTAB) { set_error("ccg_solve_batched: only CCG_BICGSTAB is batched"); return CCG_ERR_UNSUPPORTED; }
  int rc = check_block(op, nrhs, Y, ldy, X, ldx, "ccg_solve_batched");
  if (rc != CCG_OK) return static_cast<ccg_status>(rc);
  if (maxit < 0 || !(tol >= 0.0)) { set_error("ccg_solve_batched: need maxit >= 0 and tol >= 0"); return CCG_ERR_INVALID; }
  return static_cast<ccg_status>(solve_batched(h, op, nrhs, Y, ldy, X, ldx, tol, maxit, iters, status, relres));
}

ccg_status ccg_solve_batched_refined(ccg_handle* h, ccg_method method, const ccg_operator* op,
                                     const ccg_operator* op_in, int64_t nrhs, const void* Y, int64_t ldy, void* X,
                                     int64_t ldx, double tol, int max_outer, double inner_tol, int inner_maxit,
                                     int32_t* outer, int32_t* inner, int32_t* status, double* relres) {
  if (!h || !op_in) { set_error("ccg_solve_batched_refined: NULL argument"); return CCG_ERR_INVALID; }
  if (method != CCG_BICGSTAB) {
    set_error("ccg_solve_batched_refined: only CCG_BICGSTAB is batched");
    return CCG_ERR_UNSUPPORTED;
  }
  int rc = check_block(op, nrhs, Y, ldy, X, ldx, "ccg_solve_batched_refined");
  if (rc != CCG_OK) return static_cast<ccg_status>(rc);
  if (op->dtype != CCG_C128 || op_in->dtype != CCG_C64 || op_in->n != op->n || op_in->kind != CCG_OPK_DENSE) {
    set_error("ccg_solve_batched_refined: need complex128 and complex64 dense operators of the same size");
    return CCG_ERR_INVALID;
  }
  if (!(tol >= 0.0) || max_outer < 0 || !(inner_tol > 0.0) || inner_maxit < 1) {
    set_error("ccg_solve_batched_refined: need tol >= 0, max_outer >= 0, inner_tol > 0, inner_maxit >= 1");
    return CCG_ERR_INVALID;
  }
  return static_cast<ccg_status>(solve_batched_refined(h, op, op_in, nrhs, Y, ldy, X, ldx, tol, max_outer, inner_tol,
                                                       inner_maxit, outer, inner, status, relres));
}

ccg_status ccg_block_matvec(ccg_handle* h, const ccg_operator* op, int64_t nrhs, const void* X, int64_t ldx, void* Y,
                            int64_t ldy) {
  if (!h) { set_error("ccg_block_matvec: NULL handle"); return CCG_ERR_INVALID; }
  int rc = check_block(op, nrhs, X, ldx, Y, ldy, "ccg_block_matvec");
  if (rc != CCG_OK) return static_cast<ccg_status>(rc);
  return static_cast<ccg_status>(block_matvec(h, op, nrhs, X, ldx, Y, ldy));
}

// Arguments of the many-system solves: dense operators of one precision
// (ops) and, when refining, their complex64 copies (ops_in).
static int check_multi(ccg_handle* h, ccg_method method, int64_t count, const ccg_operator* const* ops,
                       const ccg_operator* const* ops_in, const void* const* y, void* const* x, const double* tol,
                       const char* who) {
  if (!h || !ops || !y || !x || !tol) { set_error(std::string(who) + ": NULL argument"); return CCG_ERR_INVALID; }
  if (method != CCG_BICGSTAB && method != CCG_CGNR && method != CCG_QMR && method != CCG_COCG) {
    set_error(std::string(who) + ": method must be BiCGSTAB, CGNR, QMR or COCG");
    return CCG_ERR_UNSUPPORTED;
  }
  const int dt = ops_in ? CCG_C64 : (count > 0 && ops[0] ? ops[0]->dtype : CCG_C128);
  const int cap = pk_capacity(h, method, dt);
  if (count < 1 || count > cap) {
    set_error(std::string(who) + ": need 1 <= count <= " + std::to_string(cap) + " (resident blocks)");
    return CCG_ERR_INVALID;
  }
  for (int64_t k = 0; k < count; ++k) {
    const ccg_operator* op = ops[k];
    if (!op || op->kind != CCG_OPK_DENSE) { set_error(std::string(who) + ": dense operators only"); return CCG_ERR_UNSUPPORTED; }
    if (op->dtype != ops[0]->dtype) { set_error(std::string(who) + ": operators of one precision"); return CCG_ERR_INVALID; }
    if (ops_in) {
      const ccg_operator* oi = ops_in[k];
      if (op->dtype != CCG_C128 || !oi || oi->kind != CCG_OPK_DENSE || oi->dtype != CCG_C64 || oi->n != op->n) {
        set_error(std::string(who) + ": need complex128 operators and complex64 copies of the same sizes");
        return CCG_ERR_INVALID;
      }
    }
    if (method == CCG_COCG && !(op->flags & CCG_OP_SYMMETRIC)) {
      set_error(std::string(who) + ": COCG needs operators flagged CCG_OP_SYMMETRIC");
      return CCG_ERR_INVALID;
    }
    const size_t esz = op->dtype == CCG_C128 ? 16 : 8;
    if (!y[k] || !x[k] || !aligned(y[k], esz) || !aligned(x[k], esz)) {
      set_error(std::string(who) + ": y and x must be aligned device vectors");
      return CCG_ERR_INVALID;
    }
    if (!(tol[k] >= 0.0)) { set_error(std::string(who) + ": need tol >= 0"); return CCG_ERR_INVALID; }
  }
  return CCG_OK;
}

ccg_status ccg_solve_multi(ccg_handle* h, ccg_method method, int64_t count, const ccg_operator* const* ops,
                           const void* const* y, void* const* x, const double* tol, int maxit, int32_t* iters,
                           int32_t* status, double* relres) {
  int rc = check_multi(h, method, count, ops, nullptr, y, x, tol, "ccg_solve_multi");
  if (rc != CCG_OK) return static_cast<ccg_status>(rc);
  if (maxit < 0) { set_error("ccg_solve_multi: need maxit >= 0"); return CCG_ERR_INVALID; }
  return static_cast<ccg_status>(solve_multi(h, method, (int)count, ops, y, x, tol, maxit, iters, status, relres));
}

ccg_status ccg_solve_multi_refined(ccg_handle* h, ccg_method inner_method, int64_t count,
                                   const ccg_operator* const* ops, const ccg_operator* const* ops_inner,
                                   const void* const* y, void* const* x, const double* tol, int max_outer,
                                   double inner_tol, int inner_maxit, int32_t* outer, int32_t* inner,
                                   int32_t* status, double* relres) {
  int rc = check_multi(h, inner_method, count, ops, ops_inner, y, x, tol, "ccg_solve_multi_refined");
  if (rc != CCG_OK) return static_cast<ccg_status>(rc);
  if (max_outer < 0 || !(inner_tol > 0.0) || inner_maxit < 1) {
    set_error("ccg_solve_multi_refined: need max_outer >= 0, inner_tol > 0, inner_maxit >= 1");
    return CCG_ERR_INVALID;
  }
  return static_cast<ccg_status>(solve_multi_refined(h, inner_method, (int)count, ops, ops_inner, y, x, tol, max_outer,
                                                     inner_tol, inner_maxit, outer, inner, status, relres));
}

ccg_status ccg_set_option(ccg_handle* h, int option, int value) {
  if (!h) { set_error("ccg_set_option: NULL handle"); return CCG_ERR_INVALID; }
  if (option == CCG_OPT_TENSOR_CORES && value >= 0 && value <= 2) {
    h->tc_mode = value;
    return CCG_OK;
  }
  if (option == CCG_OPT_TC_EXACT && (value == 0 || value == 1)) {
    h->tc_exact = value;
    return CCG_OK;
  }
  if (option == CCG_OPT_TC_SPLIT && (value == 2 || value == 3)) {
    h->tc_terms = value;
    return CCG_OK;
  }
  if (option == CCG_OPT_GMRES_RESTART && value >= 1 && value <= kMaxBasis) {
    h->gm_restart = value;
    return CCG_OK;
  }
  if (option == CCG_OPT_BICGSTAB_L && value >= 1 && value <= kMaxEll) {
    h->bicgstab_l = value;
    return CCG_OK;
  }
  if (option == CCG_OPT_PDL && (value == 0 || value == 1)) {
    h->pdl = value;
    return CCG_OK;
  }
  if (option == CCG_OPT_FP64_SWEEP && (value == 0 || value == 1)) {
    h->fx_mode = value;
    return CCG_OK;
  }
  if (option == CCG_OPT_PERSISTENT && value >= 0 && value <= 2) {
    h->persistent = value;
    return CCG_OK;
  }
  if (option == CCG_OPT_PK_BLOCKS && value >= 0 && value <= 32) {
    h->pk_blocks = value;
    return CCG_OK;
  }
  if (option == CCG_OPT_WAIT_LIMIT && value >= 0) {
    h->wait_limit = value == 0 ? (4ll << 30) : ((long long)value << 10);
    return CCG_OK;
  }
  if (option == CCG_OPT_TEST_WITHHOLD && value >= 0 && value <= 2) {
    h->test_withhold = value;
    return CCG_OK;
  }
  set_error("ccg_set_option: unknown option or value out of range");
  return CCG_ERR_INVALID;
}

ccg_status ccg_timing_enable(ccg_handle* h, int enable) {
  if (!h) return CCG_ERR_INVALID;
  if (enable && !h->skip_rec) {
    const size_t cap = (size_t)1 << 20;  // sweeps between two collections
    if (cudaMalloc(&h->skip_rec, cap * sizeof(int)) != cudaSuccess ||
        cudaMemsetAsync(h->skip_rec, 0, cap * sizeof(int), h->stream) != cudaSuccess) {
      cudaGetLastError();
      if (h->skip_rec) cudaFree(h->skip_rec);
      h->skip_rec = nullptr;
      set_error("ccg_timing_enable: allocation failed");
      return CCG_ERR_NOMEM;
    }
    h->skip_cap = cap;
  }
  h->timing = enable != 0;
  return CCG_OK;
}

ccg_status ccg_timing_read(ccg_handle* h, int dtype, int kind, int64_t* sweeps, double* total_ms,
                           double* bytes_per_sweep) {
  if (!h || kind < 0 || kind >= CCG_SWEEP_KINDS || (dtype != CCG_C64 && dtype != CCG_C128)) {
    set_error("ccg_timing_read: bad handle, dtype or kind");
    return CCG_ERR_INVALID;
  }
  API_CUDA(cudaStreamSynchronize(h->stream));
  timing_collect(h);
  const int slot = dtype * CCG_SWEEP_KINDS + kind;
  if (sweeps) *sweeps = h->timed_sweeps[slot];
  if (total_ms) *total_ms = h->timed_ms[slot];
  if (bytes_per_sweep)
    *bytes_per_sweep = h->timed_sweeps[slot] > 0 ? h->timed_bytes[slot] / (double)h->timed_sweeps[slot]
                                                 : h->bytes_per_sweep[slot];
  return CCG_OK;
}

ccg_status ccg_timing_reset(ccg_handle* h) {
  if (!h) return CCG_ERR_INVALID;
  API_CUDA(cudaStreamSynchronize(h->stream));
  timing_collect(h);
  for (int k = 0; k < 2 * CCG_SWEEP_KINDS; ++k) {
    h->timed_sweeps[k] = 0;
    h->timed_ms[k] = 0.0;
    h->timed_bytes[k] = 0.0;
  }
  return CCG_OK;
}

int64_t ccg_launch_count(const ccg_handle* h) { return h ? h->launches : 0; }

}  // extern "C"
