/*
 * ccg.h -- C ABI of libccg, GB300 (sm_103a) complex Krylov solvers.
 *
 * Problem (CCGPAK 2.0 manual, Sec. 1): solve A x = y for a complex matrix A,
 * unknown x and known right-hand side y, in single or double precision
 * (abstract; Sec. 5 `ddprecision`).  The operator is kept apart from the
 * iteration (Sec. 5: `matvec` for A x and `cmatvec` for A^H x), and the
 * solve takes a tolerance and an iteration cap (Sec. 5 `cgmodule`:
 * `epsilon_err`, `maxit`).  The methods are those of Sec. 2.1 (PIM:
 * `bicgstab`, `cgnr`, `qmr`, `bigcg`, `rgmres`, `cgs`, `cgne`, `tfqmr`), Sec. 2.2 (the
 * Sarkar complex-symmetric CG), Sec. 3.1 (BiCGstab(l)) and Sec. 3.4 (COCR), in
 * their unpreconditioned
 * textbook forms.
 *
 * Conventions shared by every entry point:
 *  - Complex vectors and matrices are interleaved (re, im) pairs in the
 *    operator's precision: CCG_C128 = two doubles (16 B per element),
 *    CCG_C64 = two floats (8 B per element).
 *  - Pointers named "device" must be CUDA device (or managed) memory that
 *    stays valid for the call; nothing is copied or freed by the library
 *    unless stated.  ccg_solve also accepts host pointers for y and x (see
 *    there).
 *  - A handle owns its CUDA stream binding and its workspace; all work is
 *    enqueued on that stream.  A handle must not be used from two host
 *    threads at once.  Calls return a ccg_status; negative values are
 *    errors, after which ccg_last_error() gives a message.
 *  - The library never falls back to host arithmetic: without a usable
 *    CUDA device every call that computes returns CCG_ERR_CUDA.
 */
#ifndef CCG_H_
#define CCG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CCG_ABI_VERSION 1

typedef enum {
  CCG_BICGSTAB = 0, /* van der Vorst BiCGSTAB (Sec. 2.1, PIM `bicgstab`)      */
  CCG_CGNR = 1,     /* CG on A^H A x = A^H y (Sec. 2.1, PIM `cgnr`)          */
  CCG_QMR = 2,      /* Freund-Nachtigal QMR, no look-ahead (Sec. 2.1 `qmr`)  */
  CCG_COCG = 3,     /* complex-symmetric CG, unconjugated form (Sec. 2.2)    */
  CCG_COCR = 4,     /* Sogabe-Zhang conjugate A-orthogonal CR (Sec. 3.4)     */
  CCG_BICG = 5,     /* Fletcher BiCG with A^H, shadow r~0 = r0 (Sec. 2.1
                       PIM `bigcg`)                                         */
  CCG_GMRES = 6,    /* restarted GMRES(m) (Sec. 2.1 PIM `rgmres`); m set by
                       ccg_set_option(CCG_OPT_GMRES_RESTART), default 30    */
  CCG_CGS = 7,      /* Sonneveld CGS, shadow r^ = r0 (Sec. 2.1 PIM `cgs`)    */
  CCG_CGNE = 8,     /* Craig's CG on A A^H u = y, x = A^H u (PIM `cgne`)     */
  CCG_TFQMR = 9,    /* Freund TFQMR, two half-steps per iteration; residual
                       = the quasi-residual bound (Sec. 2.1 PIM `tfqmr`)     */
  CCG_BICGSTABL = 10 /* vanilla BiCGstab(l) (Sec. 3.1); an iteration is one
                       cycle of l BiCG steps (2 l products); l set by
                       ccg_set_option(CCG_OPT_BICGSTAB_L), default 2        */
} ccg_method;

typedef enum { CCG_C64 = 0, CCG_C128 = 1 } ccg_dtype;

typedef enum {
  CCG_OK = 0,             /* converged: ||r_k|| / ||y|| <= tol              */
  CCG_NOT_CONVERGED = 1,  /* maxit iterations done without meeting tol      */
  CCG_BREAKDOWN = 2,      /* a divisor vanished; see ccg_info.breakdown     */
  CCG_ERR_INVALID = -1,   /* bad argument                                   */
  CCG_ERR_NOMEM = -2,     /* device allocation failed                       */
  CCG_ERR_CUDA = -3,      /* CUDA runtime error or no device                */
  CCG_ERR_NONFINITE = -4, /* NaN or Inf in y or in a residual               */
  CCG_ERR_TIMEOUT = -5,   /* a bounded device wait expired                  */
  CCG_ERR_UNSUPPORTED = -6 /* method/operator combination not available     */
} ccg_status;

/* Which scalar vanished on CCG_BREAKDOWN. */
typedef enum {
  CCG_BD_NONE = 0, CCG_BD_RHO = 1, CCG_BD_SIGMA = 2, CCG_BD_TT = 3, CCG_BD_OMEGA = 4,
  CCG_BD_GAMMA = 5, CCG_BD_WW = 6, CCG_BD_XI = 7, CCG_BD_DELTA = 8, CCG_BD_EPS = 9,
  CCG_BD_BETA = 10, CCG_BD_MU = 11,
  CCG_BD_HESS = 12 /* GMRES: a zero Hessenberg column (singular projected system) */
} ccg_breakdown;

/* Operator flags. */
#define CCG_OP_SYMMETRIC 1 /* caller asserts A = A^T (required by CCG_COCG, CCG_COCR) */

typedef struct ccg_handle ccg_handle;
typedef struct ccg_operator ccg_operator;

/* Result of one solve. */
typedef struct {
  int32_t iters;       /* completed iterations (BiCGSTAB's half-step exit counts as one) */
  int32_t status;      /* ccg_status of the solve                                        */
  int32_t breakdown;   /* ccg_breakdown                                                 */
  int32_t reserved;
  double relres;       /* last recurrence residual ||r_k|| / ||y||                      */
  double true_relres;  /* ||y - A x|| / ||y|| recomputed from x at the end (-1 if skipped) */
  double ynorm;        /* ||y||_2                                                        */
} ccg_info;

/* Create a handle bound to `stream` (a cudaStream_t; NULL = legacy default
 * stream) on the current CUDA device.  *h receives the handle.  Returns
 * CCG_ERR_CUDA when no device is usable.  The environment variable
 * CCG_PHASE_MIN_ELEMS (1..64, read here) sets a floor on the vector elements
 * per thread of the fused update kernels of single-right-hand-side solves
 * (a tuning override; default 1). */
ccg_status ccg_create(ccg_handle** h, void* stream);
/* Destroy a handle and free its workspace (after synchronising its stream). */
ccg_status ccg_destroy(ccg_handle* h);
/* Rebind the handle to another stream. */
ccg_status ccg_set_stream(ccg_handle* h, void* stream);
/* Text of the last error recorded on this thread (never NULL). */
const char* ccg_last_error(void);
/* Text for a status code (never NULL). */
const char* ccg_status_string(int status);
/* Returns CCG_ABI_VERSION. */
int ccg_abi_version(void);

/* Dense operator on a caller-owned device matrix (the manual's `matvec` and
 * `cmatvec`, Sec. 5, for a dense A).  A is n x n, row-major with leading
 * dimension lda >= n, element (i, j) at A[i * lda + j], in precision `dtype`.
 * The matrix is NOT copied: it must stay valid and unchanged while the
 * operator is used.  flags: CCG_OP_SYMMETRIC or 0.  Errors: CCG_ERR_INVALID
 * for n < 1, lda < n, a NULL pointer, or A not 8-byte (C64) / 16-byte
 * (C128) aligned. */
ccg_status ccg_op_dense(ccg_handle* h, ccg_dtype dtype, int64_t n, const void* A, int64_t lda, int flags,
                        ccg_operator** op);
/* Discrete-dipole operator (the DDSCAT application named in Sec. 1; the
 * manual does not define it -- this is the standard system):
 *   (A p)_s = p_s / alpha - sum_{t != s} G(r_s - r_t) p_t
 * over the occupied cells of an nx x ny x nz lattice with unit spacing,
 * G(r) = exp(ikr)/r^3 [ (kr)^2 (I - u u^T) + (1 - ikr)(3 u u^T - I) ] the
 * field tensor of a point dipole (u = r/|r|, k = kd), and the
 * Clausius-Mossotti polarizability alpha = (3/4pi)(m^2 - 1)/(m^2 + 2) for
 * refractive index m = m_re + i m_im.
 *  occ   host array of nx*ny*nz bytes, occ[(i*ny + j)*nz + l] != 0 marks an
 *        occupied cell; read during the call only.
 * Unknowns: 3N for N occupied cells, ordered v[a*N + s] (a = x, y, z; sites
 * in occ order).  The operator is complex symmetric (flagged
 * CCG_OP_SYMMETRIC).  It is applied by zero-padded FFT convolution on a
 * (2nx) x (2ny) x (2nz) grid in the operator's precision; each of 2nx, 2ny,
 * 2nz must be of the form 2^a 3^b and at most 256 (else CCG_ERR_INVALID).
 * The operator owns its device memory (field tensor, FFT grids): about
 * 9 * 8 nx ny nz * (16 B complex128 | 8 B complex64); its applications use
 * one set of grids, so they must not run concurrently on two streams.
 * Synchronises the handle's stream. */
ccg_status ccg_op_dipole(ccg_handle* h, ccg_dtype dtype, int nx, int ny, int nz, const uint8_t* occ, double kd,
                         double m_re, double m_im, ccg_operator** op);
/* Number of occupied sites N of a dipole operator (0 for other operators). */
int64_t ccg_dipole_sites(const ccg_operator* op);
/* A user-supplied operator: the manual's `matvec` and `cmatvec` (Sec. 5),
 * kept apart from the iteration.  Each is a host function that ENQUEUES
 *   y = A x   (matvec)   or   y = A^H x   (cmatvec)
 * on `stream` (the handle's cudaStream_t) for device vectors x and y of n
 * complex values in the operator's precision (interleaved re, im; 16-byte
 * aligned), and returns 0 on success.  The library calls it from the thread
 * that runs the solve, possibly a few iterations ahead of the GPU and,
 * near the end of a solve, for products whose results are not used; x and
 * y are library workspace that stays valid until the enqueued work has run.
 * It must not synchronise with work it has not enqueued itself on `stream`,
 * and must not call the handle that invoked it.  A nonzero return ends the
 * solve with CCG_ERR_CUDA (the message names the callback). */
typedef int (*ccg_matvec_fn)(void* ctx, int64_t n, const void* x, void* y, void* stream);
/* Operator from callbacks (see ccg_matvec_fn); ctx is passed through.
 * cmatvec may be NULL: the methods that need A^H (CGNR, QMR, BiCG, CGNE)
 * then return CCG_ERR_UNSUPPORTED.  flags: CCG_OP_SYMMETRIC or 0.  Usable
 * with ccg_matvec, ccg_solve and ccg_solve_refined (either operator); the
 * batched solves and ccg_block_matvec need a dense operator.  Errors:
 * CCG_ERR_INVALID for n < 1, a NULL matvec or unknown flags. */
ccg_status ccg_op_callback(ccg_handle* h, ccg_dtype dtype, int64_t n, ccg_matvec_fn matvec, ccg_matvec_fn cmatvec,
                           void* ctx, int flags, ccg_operator** op);
/* Free an operator (not the caller's matrix).  A dense operator's
 * tensor-core copies (split-bf16 terms, digit slices: made by its first
 * block product of each kind, on that call's stream) are freed in stream
 * order on the stream that made them, so an operator must be destroyed
 * before that stream is.  Calls on other streams that use the operator
 * after such a first call must be ordered after it (synchronise that
 * call's stream, or wait on an event recorded after it). */
ccg_status ccg_op_destroy(ccg_operator* op);
/* Number of unknowns of an operator. */
int64_t ccg_op_size(const ccg_operator* op);

/* y = A x (trans = 0) or y = A^H x (trans = 1): the manual's `matvec` /
 * `cmatvec` (Sec. 5).  x and y are device vectors of ccg_op_size(op)
 * elements in the operator's precision; they must not overlap.  Enqueued on
 * the handle's stream; returns without synchronising. */
ccg_status ccg_matvec(ccg_handle* h, const ccg_operator* op, int trans, const void* x, void* y);

/* Dot product of two device vectors of n elements, the Fortran
 * `dot_product` of the manual (Sec. 1, Sec. 2.1): conj = 1 gives
 * <u, v> = sum conj(u_i) v_i, conj = 0 gives [u, v] = sum u_i v_i.  The sum
 * is accumulated in double; out2 (host) receives {re, im}.  Synchronises
 * the handle's stream. */
ccg_status ccg_dot(ccg_handle* h, ccg_dtype dtype, int64_t n, const void* u, const void* v, int conj,
                   double* out2);

/* Solve A x = y with `method` (Sec. 1 problem statement, Sec. 2 methods).
 *  y        right-hand side, n elements; never written.
 *  x        on entry the start vector x0, on exit the solution (the last
 *           iterate also on CCG_NOT_CONVERGED / CCG_BREAKDOWN).
 *           y and x may both be device pointers or both host pointers; with
 *           host pointers the library copies them through its workspace.
 *  tol      stop when ||r_k||_2 / ||y||_2 <= tol on the recurrence residual.
 *  maxit    iteration cap (>= 0).
 *  res_hist optional host array of maxit + 1 doubles: res_hist[k] =
 *           ||r_k|| / ||y|| for k = 0 .. iters; may be NULL.
 *  info     optional host struct receiving the result; info->true_relres is
 *           computed (one extra operator application) only when info is not
 *           NULL.
 * y = 0 gives x = 0, iters = 0, CCG_OK.  CCG_COCG and CCG_COCR need an
 * operator made with CCG_OP_SYMMETRIC (else CCG_ERR_INVALID).  Products per
 * iteration: BiCGSTAB, CGS, TFQMR, CGNR and CGNE two, BiCGstab(l) 2 l; QMR
 * and BiCG A p and A^H q
 * (one read of a dense A); COCG, COCR and GMRES one.  Blocks the calling thread
 * until the solve has finished on the handle's stream.  Returns the solve's
 * status (CCG_OK, CCG_NOT_CONVERGED, CCG_BREAKDOWN) or an error. */
ccg_status ccg_solve(ccg_handle* h, ccg_method method, const ccg_operator* op, const void* y, void* x, double tol,
                     int maxit, double* res_hist, ccg_info* info);

/* Mixed-precision solve of A x = y: iterative refinement with the residual
 * r = y - A x and the update x += d in complex128, and each correction
 * A d = r solved by `inner_method` in complex64 (the manual's single and
 * double precision, abstract and Sec. 5, used together).
 *  op        complex128 operator of A (residuals, updates)
 *  op_inner  complex64 operator of the same matrix rounded to single
 *            precision (the inner Krylov sweeps); same size as op
 *  y, x      complex128 right-hand side and start/solution, both device or
 *            both host pointers (as in ccg_solve)
 *  tol       stop when ||y - A x|| / ||y|| <= tol, the residual recomputed
 *            in complex128 from x at every outer step
 *  max_outer cap on corrections (>= 0)
 *  inner_tol, inner_maxit  relative tolerance (> 0) and cap (>= 1) of each
 *            inner solve
 *  res_hist  optional host array of max_outer + 1 doubles: the outer
 *            residuals ||y - A x_j|| / ||y||, j = 0 .. info->iters
 *  inner_iters optional: total inner iterations
 *  info      optional; iters = corrections applied, relres = true_relres =
 *            the last outer residual.
 * Returns CCG_OK, CCG_NOT_CONVERGED (max_outer reached), CCG_BREAKDOWN (an
 * inner solve broke down before its first iteration) or an error. */
ccg_status ccg_solve_refined(ccg_handle* h, ccg_method inner_method, const ccg_operator* op,
                             const ccg_operator* op_inner, const void* y, void* x, double tol, int max_outer,
                             double inner_tol, int inner_maxit, double* res_hist, int* inner_iters, ccg_info* info);

/* Many right-hand sides at once (the Sec. 1 problem for a block Y of k
 * columns): BiCGSTAB (Sec. 2.1) per column, all columns advancing together so
 * that each iteration's two operator applications are block products A P,
 * A S that read the matrix once for all columns.  Every column keeps its own
 * scalars, iteration count and stopping test (||r_c|| / ||y_c|| <= tol); a
 * stopped column is frozen while the others continue.
 *  method    CCG_BICGSTAB (others return CCG_ERR_UNSUPPORTED)
 *  op        dense operator (CCG_ERR_UNSUPPORTED otherwise)
 *  nrhs      k, 1 <= k <= 256
 *  Y, ldy    device block, column c at Y + c*ldy (ldy >= n), op's precision
 *  X, ldx    device block, start vectors in, solutions out
 *  iters, status, relres  optional host arrays of k entries
 * Returns the worst column status (an error, else CCG_BREAKDOWN >
 * CCG_NOT_CONVERGED > CCG_OK).  Synchronises the handle's stream. */
ccg_status ccg_solve_batched(ccg_handle* h, ccg_method method, const ccg_operator* op, int64_t nrhs, const void* Y,
                             int64_t ldy, void* X, int64_t ldx, double tol, int maxit, int32_t* iters,
                             int32_t* status, double* relres);

/* Batched mixed precision: complex128 block residuals R = Y - A X and
 * updates X += D, each correction A D = R solved by the batched complex64
 * BiCGSTAB above (op_inner: the complex64 copy of op's matrix).  Y, X are
 * complex128.  X0 = 0 is detected on the device and its product skipped.
 * Columns stop refining individually when ||y_c - A x_c|| / ||y_c|| <= tol
 * (recomputed in complex128).  outer, inner: optional host arrays of k
 * entries (corrections, inner iterations in total).  Other arguments as in
 * ccg_solve_batched and ccg_solve_refined. */
ccg_status ccg_solve_batched_refined(ccg_handle* h, ccg_method inner_method, const ccg_operator* op,
                                     const ccg_operator* op_inner, int64_t nrhs, const void* Y, int64_t ldy, void* X,
                                     int64_t ldx, double tol, int max_outer, double inner_tol, int inner_maxit,
                                     int32_t* outer, int32_t* inner, int32_t* status, double* relres);

/* Many independent systems A_k x_k = y_k (the Sec. 1 problem, k = 0 ..
 * count-1) of uneven sizes, solved together in one cooperative launch: the
 * GPU's resident blocks are split into one group per system, in proportion
 * to its matrix bytes (every system at least one block), and each group runs
 * its system's iteration with barriers among its own blocks only, so
 * systems of different sizes and iteration counts advance independently.  A
 * system's result is bitwise that of ccg_solve with CCG_OPT_PERSISTENT = 0
 * (the same sweeps and fused updates, reduced in the same order).  Meant for
 * small systems, whose solves are otherwise bound by launch latency.
 *  method    CCG_BICGSTAB, CCG_CGNR, CCG_QMR or CCG_COCG (else
 *            CCG_ERR_UNSUPPORTED)
 *  count     1 .. the resident blocks of the launch (about 3 per SM)
 *  ops       count dense operators of one precision (COCG: flagged
 *            CCG_OP_SYMMETRIC); the same operator may appear more than once
 *  y, x      count device vectors each (x: start vector in, solution out)
 *  tol       count relative residual targets
 *  maxit     iteration cap of every system
 *  iters, status, relres  optional host arrays of count entries: iterations,
 *            ccg_status, and ||y - A x|| / ||y|| recomputed from x
 * Returns the worst status (an error, else CCG_BREAKDOWN > CCG_NOT_CONVERGED
 * > CCG_OK); CCG_ERR_TIMEOUT if a group barrier gave up (CCG_OPT_WAIT_LIMIT).
 * Synchronises the handle's stream. */
ccg_status ccg_solve_multi(ccg_handle* h, ccg_method method, int64_t count, const ccg_operator* const* ops,
                           const void* const* y, void* const* x, const double* tol, int maxit, int32_t* iters,
                           int32_t* status, double* relres);
/* The same with mixed precision (as ccg_solve_refined, per system): each
 * outer step is one launch over the systems still refining -- x += d, the
 * residual r = y - A x in complex128 and its test -- and one launch of their
 * complex64 corrections A d = r.  ops: complex128 operators; ops_inner:
 * complex64 operators of the same matrices.  outer, inner: optional host
 * arrays (corrections applied, inner iterations in total); relres: the last
 * complex128 residual of each system.  Other arguments as above and in
 * ccg_solve_refined. */
ccg_status ccg_solve_multi_refined(ccg_handle* h, ccg_method inner_method, int64_t count,
                                   const ccg_operator* const* ops, const ccg_operator* const* ops_inner,
                                   const void* const* y, void* const* x, const double* tol, int max_outer,
                                   double inner_tol, int inner_maxit, int32_t* outer, int32_t* inner,
                                   int32_t* status, double* relres);

/* Y = A X for a block of right-hand sides: the manual's `matvec` (Sec. 5)
 * applied to nrhs columns at once.  X, Y: device column-major blocks of the
 * operator's precision (column c at X + c*ldx; ldx, ldy >= n), 1 <= nrhs <=
 * 256; dense operators only.  complex64 products run on the tensor cores
 * (split-bf16 operands, fp32 accumulation; see CCG_OPT_TC_SPLIT) unless
 * disabled with ccg_set_option(h, CCG_OPT_TENSOR_CORES, 0); complex128
 * products, and complex64 ones with that option off, run on the tensor
 * cores as exact integer products of seven-bit digit slices
 * (CCG_OPT_TC_EXACT: FP64-accurate for complex128, FP32-accurate for
 * complex64) for n divisible by 4 and n <= 32768; other products use CUDA
 * cores.  Synchronises the stream; returns CCG_ERR_TIMEOUT if a bounded wait
 * of a tensor-core pipeline gave up. */
ccg_status ccg_block_matvec(ccg_handle* h, const ccg_operator* op, int64_t nrhs, const void* X, int64_t ldx, void* Y,
                            int64_t ldy);

/* Handle options.
 * CCG_OPT_TENSOR_CORES selects where complex64 block products run on the
 * tcgen05 tensor cores: 0 never; 1 (default) in ccg_block_matvec and in the
 * inner solves of ccg_solve_batched_refined; 2 also in plain complex64
 * ccg_solve_batched.
 * CCG_OPT_TC_SPLIT: bf16 terms per operand entry, 2 (default: three
 * products) or 3 (six products).  The tensor cores' fp32 accumulation bounds
 * both to ~1e-5 relative at K ~ 10^3 and ~1e-4 at K ~ 10^4, so the third
 * term rarely pays; refined batched solves correct the difference with one
 * exact complex64 residual per correction.
 * CCG_OPT_GMRES_RESTART: the cycle length m of CCG_GMRES, 1..64 (default
 * 30); the solve holds m + 1 basis vectors in the handle's workspace.
 * CCG_OPT_BICGSTAB_L: the degree l of CCG_BICGSTABL, 1..4 (default 2).
 * CCG_OPT_TC_EXACT: 1 (default) runs the block products that must be
 * accurate in their own precision -- every complex128 one (batched
 * complex128 solves, the residuals of refined batched solves,
 * ccg_block_matvec) and the complex64 ones that do not take the split-bf16
 * path (the exact complex64 residuals of refined batched solves, plain
 * complex64 batched solves) -- on the tensor cores by the integer-slice
 * scheme: each row of A and column of X is scaled by a power of two and cut
 * into S signed 7-bit digits (S = 8 for complex128, 4 for complex64), the
 * digit pairs of S significance levels are summed exactly by bf16 MMAs with
 * fp32 accumulation and combined in int64.  The result is as accurate as a
 * GEMM in the operands' precision (error ~ K 2^-53, resp. K 2^-24, times
 * max|a| max|x| per entry).  0 uses CUDA cores for them.
 * CCG_OPT_PERSISTENT selects how ccg_solve and the inner solves of
 * ccg_solve_refined run BiCGSTAB, CGNR, QMR or COCG on a dense operator: 1 as
 * one cooperative launch per solve (the iteration's sweeps and fused updates
 * back to back inside the kernel, separated by grid barriers); 0 as the
 * kernel-per-step loop, which every other method and operator uses; 2 (the
 * default) as the library's tuned table says for the precision, method and
 * order (measured on GB300 by the package's autotune.py).  Both forms run
 * the same arithmetic in the same order: results are bitwise equal.
 * CCG_OPT_PK_BLOCKS: resident blocks per SM of that launch, 1..32 (0, the
 * default: the tuned value, else the occupancy limit).
 * CCG_OPT_WAIT_LIMIT: the bounded wait of the persistent launch's barriers,
 * in units of 1024 SM clock cycles (0: the default, 2^22 units, about 2 s at
 * 2 GHz).  A block that waits longer gives up, the call returns
 * CCG_ERR_TIMEOUT and the handle stays usable.
 * CCG_OPT_FP64_SWEEP selects how y = A x runs for a complex128 dense
 * operator: 1 (default) in 53-bit fixed point on the integer pipe -- each row
 * of A and the vector scaled by its largest power of two and cut into two
 * 26-bit digits, the products summed exactly in 64-bit integers -- reading a
 * digit copy of A that the operator makes on its first such product (16
 * bytes per entry, freed with the operator; a matrix with a non-finite entry
 * keeps the FP64 pipe); error <= 2.5 n 2^-52 max_j|a_ij| max_j|x_j| per entry
 * (times the powers of two above those maxima); 0 on the FP64 pipe (FMA,
 * error ~ n 2^-53 sum_j |a_ij||x_j|).  GB300's FP64 pipe holds that sweep to a
 * third of HBM bandwidth; the integer form runs near it.
 * CCG_OPT_PDL: 1 (default) launches the kernels of the kernel-per-step loop
 * with programmatic dependent launch (each starts launching while the one
 * before finishes and waits for it inside); 0 plain stream order.  Results
 * are the same either way.
 * CCG_OPT_TEST_WITHHOLD: test hook (use with a small CCG_OPT_WAIT_LIMIT);
 * 1 makes one block of the next persistent launches leave without arriving
 * at the first barrier, and the tensor-core products' TMA producers issue no
 * copies, so that the waits on them expire; 2 makes the first K range of the
 * split-bf16 product keep its partial tile unpublished, so that the CTA
 * finishing that tile waits in vain; 0 (default) off.
 * ccg_set_option returns CCG_ERR_INVALID (and leaves the handle unchanged)
 * for a NULL handle, an unknown option or a value out of range; options
 * apply to the handle's later calls. */
#define CCG_OPT_TENSOR_CORES 1
#define CCG_OPT_TC_SPLIT 2
#define CCG_OPT_GMRES_RESTART 3
#define CCG_OPT_BICGSTAB_L 4
#define CCG_OPT_TC_EXACT 5
#define CCG_OPT_PERSISTENT 6
#define CCG_OPT_PK_BLOCKS 7
#define CCG_OPT_WAIT_LIMIT 8
#define CCG_OPT_TEST_WITHHOLD 9
#define CCG_OPT_FP64_SWEEP 10
#define CCG_OPT_PDL 11
ccg_status ccg_set_option(ccg_handle* h, int option, int value);

/* ---------------------------------------------------------------------------
 * Serving: a queue of solve requests of mixed sizes, admitted to worker slots
 * as slots and device memory (an HBM budget) free up.  Each slot owns a
 * handle and a CUDA stream, so admitted requests' work overlaps on the GPU;
 * a request's Krylov state stays resident on its slot until it finishes.
 * Requests are synthetic problems generated on the device from a seed with
 * the counter-based Philox4x32-10 generator (Salmon et al., SC'11):
 *  - CCG_REQ_DENSE: A = (shift + 0.5 + 0.5i) I + G / sqrt(n), G complex
 *    normal; nrhs complex-normal right-hand sides (the Sec. 1 problem);
 *  - CCG_REQ_DIPOLE: the discrete-dipole operator of an L^3 inscribed sphere
 *    (see ccg_op_dipole) with the x-polarised plane wave along z.
 * Precision follows the tolerance: tol >= 1e-5 runs complex64 solves,
 * smaller tol the mixed-precision refinement (complex128 residuals: a
 * complex64 residual carries ~1e-6 relative rounding on these operators and
 * cannot certify tighter tolerances).  Dense
 * requests use BiCGSTAB (batched when nrhs > 1); dipole requests COCG.
 * -------------------------------------------------------------------------- */
typedef struct ccg_server ccg_server;

#define CCG_REQ_DENSE 0
#define CCG_REQ_DIPOLE 1

typedef struct {
  int32_t kind;      /* CCG_REQ_DENSE or CCG_REQ_DIPOLE                         */
  int32_t nrhs;      /* dense: right-hand sides, 1 .. 256                      */
  int64_t n;         /* dense: matrix order                                     */
  double shift;      /* dense: diagonal shift                                   */
  uint64_t seed;     /* dense: generator seed (matrix and right-hand sides)     */
  int32_t L;         /* dipole: lattice edge (2L must be 2^a 3^b, <= 256)       */
  int32_t maxit;     /* iteration cap of each (inner) solve                     */
  double kd, m_re, m_im; /* dipole: wavenumber x spacing, refractive index      */
  double tol;        /* relative residual target                                */
  int32_t keep_x;    /* 1: keep the solution for ccg_server_wait to copy out   */
  int32_t mode;      /* 0: precision by tolerance (above); 1: plain complex128
                        solves, one right-hand side at a time (a baseline)     */
} ccg_request;

typedef struct {
  int32_t status;    /* worst column status (ccg_status)                        */
  int32_t iters;     /* largest iteration count (corrections for refinement)    */
  double relres;     /* largest final relative residual                         */
  double t_submit, t_start, t_done; /* seconds on the server's steady clock     */
  int64_t n;         /* unknowns per right-hand side                            */
  int32_t nrhs;
  int32_t slot;      /* worker slot that ran the request                        */
} ccg_result;

/* Create a server on CUDA device `device` with `slots` workers (1..32) and
 * an HBM budget in bytes for admitted requests (0: 120 GB).  Returns once
 * every slot has its stream and handle, so slot set-up is not part of any
 * request's latency. */
ccg_status ccg_server_create(ccg_server** s, int device, int slots, uint64_t hbm_budget_bytes);
/* Queue a request; *ticket identifies it.  Never blocks on the GPU. */
ccg_status ccg_server_submit(ccg_server* s, const ccg_request* req, int64_t* ticket);
/* *done = 1 once the request has finished. */
ccg_status ccg_server_poll(ccg_server* s, int64_t ticket, int* done);
/* Block until the request has finished; fill *res.  With keep_x set and x
 * non-NULL, copy the solution (n * nrhs complex values, column-major,
 * complex128) into the host buffer x and release it. */
ccg_status ccg_server_wait(ccg_server* s, int64_t ticket, ccg_result* res, void* x);
/* Seconds on the server's clock (the clock of ccg_result times). */
double ccg_server_now(const ccg_server* s);
/* Batching of small dense requests: a slot that takes a single-right-hand-
 * side dense request of order <= max_n (precision by tolerance, mode 0) also
 * takes every other such request waiting in the queue, in queue order, up to
 * max_systems (and the launch's resident blocks) and as long as their bytes
 * fit the budget, and solves them in one ccg_solve_multi_refined launch per
 * step.  Requests with several right-hand sides keep the per-slot block
 * solver, which reads the matrix once for all of them.  max_n = 0 turns it
 * off.  Default: max_n 2048, max_systems 256.  CCG_ERR_INVALID for a NULL
 * server, max_n < 0 or max_systems < 1. */
ccg_status ccg_server_set_batching(ccg_server* s, int64_t max_n, int max_systems);
/* Device bytes the admission test charges for a request: its matrices,
 * blocks and workspace while it runs, and for a dipole request its
 * operators, which the slot that ran it keeps cached (and charged) until
 * the server is destroyed.  CCG_ERR_INVALID for NULL or a bad kind. */
ccg_status ccg_server_estimate(const ccg_request* req, uint64_t* bytes);
/* Bytes currently charged against the server's budget (running requests
 * and cached operators). */
ccg_status ccg_server_charged(ccg_server* s, uint64_t* bytes);
/* Finish queued work, stop the workers and free everything. */
ccg_status ccg_server_destroy(ccg_server* s);

/* Kinds of operator sweep, for timing. */
typedef enum {
  CCG_SWEEP_N = 0,    /* y = A x                          */
  CCG_SWEEP_C = 1,    /* y = A^H x                        */
  CCG_SWEEP_BOTH = 2, /* A p and A^H q from one read of A */
  CCG_SWEEP_BLOCK = 3, /* A X for a block of right-hand sides (CUDA cores) */
  CCG_SWEEP_BLOCK_TC = 4, /* A X for a block on the tensor cores, split bf16 */
  CCG_SWEEP_BLOCK_EXACT = 5, /* A X for a block on the tensor cores, exact
                                integer digit slices */
  CCG_SWEEP_PERSIST = 6, /* a persistent solve's launch, counted as the
                            sweeps it ran (see CCG_OPT_PERSISTENT) */
  CCG_SWEEP_KINDS = 7
} ccg_sweep_kind;

/* Per-kernel timing of the operator sweeps: when enabled, each sweep that a
 * call of this handle launches is bracketed by CUDA events on the handle's
 * stream.  ccg_timing_read returns, for one precision (ccg_dtype) and one
 * sweep kind, the number of sweeps timed since the last reset, their total
 * device milliseconds, and the algorithmic bytes of one sweep (the matrix
 * bytes read).  It synchronises the handle's stream.  ccg_timing_reset
 * synchronises the stream and sets every count and total to zero.  All three
 * return CCG_ERR_INVALID for a NULL handle (ccg_timing_read also for a bad
 * dtype or kind). */
ccg_status ccg_timing_enable(ccg_handle* h, int enable);
ccg_status ccg_timing_read(ccg_handle* h, int dtype, int kind, int64_t* sweeps, double* total_ms,
                           double* bytes_per_sweep);
ccg_status ccg_timing_reset(ccg_handle* h);

/* Number of kernels this handle has launched since it was created. */
int64_t ccg_launch_count(const ccg_handle* h);

/* Measured issue rate of one arithmetic pipe on the handle's device, in
 * giga-operations per second (one fused multiply-add = one operation):
 * pipe 0 = FP64 fused multiply-add (the pipe of the complex128 sweeps on
 * FP64), 1 = FP32 fused multiply-add, 2 = 32 x 32 -> 64-bit integer
 * multiply-add as the compiler selects it (the form of the fixed-point
 * complex128 sweeps), 3 and 4 = the same through the PTX forms mad.wide.s32
 * and mad.lo.cc.u32 + madc.hi.s32 (which the GB300 issues to different
 * pipes).  Runs six
 * launches of about 10 ms on the handle's stream and synchronises it; the
 * median of five timed launches is returned.  It is the denominator of the
 * arithmetic-bound rooflines (the paper has no counterpart).  Returns
 * CCG_ERR_INVALID for a NULL handle or output pointer or a pipe outside
 * 0..4, CCG_ERR_CUDA when a CUDA call fails. */
ccg_status ccg_pipe_rate(ccg_handle* h, int pipe, double* gops);

/* Host-side check of the work split of the complex64 block product on the
 * tensor cores (diagnostic; no device work, no GPU needed; the paper has no
 * counterpart).  For an n x n operator, k right-hand sides, `terms` bf16
 * terms (2 or 3) and `sms` SMs it runs the cut that the product's launcher
 * and kernel use -- the R = row blocks x K blocks units cut into equal
 * ranges, one CTA per range and column tile -- and verifies: every (row
 * block, column tile, K block) is computed exactly once and lies inside the
 * operator; every output tile has one finishing CTA; a CTA leaves at most its
 * first segment unfinished; the CTAs a finisher waits for are lower-numbered
 * and their unfinished pieces are exactly the tile's earlier K blocks; their
 * partial-tile and flag indexes stay inside the buffers sized for the launch.
 * *ctas receives the launch's CTA count, *bad the number of violations (0
 * when the cut is sound).  CCG_ERR_INVALID for n < 1, k outside 1..256,
 * terms other than 2 or 3, sms < 1 or a NULL output; CCG_ERR_NOMEM when the
 * host bookkeeping cannot be allocated. */
ccg_status ccg_check_block_schedule(int64_t n, int k, int terms, int sms, int* ctas, int64_t* bad);

/* Allocation-free y = A^H x for a dense matrix.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory -- for instance a host program whose device memory is all
 * owned by its own pool allocator, or a loop that cannot afford the
 * device-wide synchronisation that cudaMalloc / cudaFree imply.  Every other
 * call of this library needs a handle, whose workspace is allocated with
 * cudaMalloc; this one needs none and calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 * Arguments are those of ccg_op_dense + ccg_matvec(trans = 1): A is n x n,
 * row-major with leading dimension lda, precision `dtype`, on the current
 * CUDA device; x (input) and y (output) are device vectors of n elements;
 * the work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 * stream) and the call returns without synchronising.
 *
 * Scratch: the partial sums live in one fixed device array of
 * CCG_NOALLOC_SCRATCH_BYTES inside the library, resident on each device
 * from the first ccg_matvec_h_noalloc call there (or from library load
 * under eager module loading) until the process exits.  n above CCG_NOALLOC_MAX_N is
 * rejected with CCG_ERR_INVALID before anything is launched.  All calls on a
 * device share that array, so two calls whose work overlaps on the GPU (on
 * different streams, or from different threads) race and give wrong results:
 * order them on one stream or synchronise between them.  Each call writes
 * every scratch entry it reads, so nothing carries over from the last call.
 * The first call on each device looks up the array's device address (with
 * that device current) and loads every kernel the entry point uses (both
 * precisions); make that first call before any stream capture.
 * Returns CCG_OK, CCG_ERR_INVALID (NULL or misaligned pointer, bad dtype,
 * n < 1, lda < n, n too large) or CCG_ERR_CUDA (no device, launch error). */
#define CCG_NOALLOC_MAX_N 65536
#define CCG_NOALLOC_SCRATCH_BYTES (16u << 20)
ccg_status ccg_matvec_h_noalloc(ccg_dtype dtype, int64_t n, const void* A, int64_t lda, const void* x, void* y,
                                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CCG_H_ */
