// Host-side structures of libccg shared by its translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ccg.h"

namespace ccg {
struct SolveState;
void set_error(const std::string& msg);
}  // namespace ccg

enum { CCG_OPK_DENSE = 0, CCG_OPK_DIPOLE = 1, CCG_OPK_CALLBACK = 2 };

// Device data of a discrete-dipole operator (owned by the operator).
struct DipoleData {
  int nx = 0, ny = 0, nz = 0;   // lattice box
  int64_t nsites = 0;           // occupied sites N; unknowns 3N
  double kd = 0.0;              // wavenumber times lattice spacing
  double alpha_inv[2] = {0.0, 0.0};
  int* idx = nullptr;           // site number of each lattice cell, or -1
  void* work = nullptr;         // 3 FFT grids
  void* ghat = nullptr;         // octant (0..M/2 per axis) of the 6 transformed field-tensor components
  void* tw[3] = {nullptr, nullptr, nullptr};  // twiddle tables along x, y, z
  int bl = 8;                   // lines per block of the FFT passes
  double sweep_bytes = 0.0;     // algorithmic bytes of one application
  int kernels = 5;              // kernels per application (3 when the z and y passes are fused)
};

struct ccg_operator {
  int kind = CCG_OPK_DENSE;
  ccg_dtype dtype = CCG_C128;
  int64_t n = 0;
  int flags = 0;
  // dense
  const void* A = nullptr;
  int64_t lda = 0;
  int unit = 1;  // complex numbers per 16-byte load (2 only for aligned complex64 with even n, lda)
  // dipole
  DipoleData dip;
  // user callbacks (the manual's matvec / cmatvec)
  ccg_matvec_fn cb_matvec = nullptr;
  ccg_matvec_fn cb_cmatvec = nullptr;
  void* cb_ctx = nullptr;
  // tensor-core copies of a complex64 dense matrix (made on first use)
  bool tc_ready = false;
  int tc_terms = 0;                            // bf16 terms per entry (2 or 3)
  void* tc_ahi = nullptr;                      // the terms, one n x 2n bf16 matrix each
  cudaStream_t tc_stream = nullptr;            // stream they were allocated (and are freed) on
  alignas(64) unsigned char tc_map[3][128] = {};  // their TMA descriptors
  // integer digit slices of a dense matrix for the exact tensor-core product
  // (made on first use): 8 (complex128) or 4 (complex64) n x 2n bf16
  // slices, then the row exponents
  bool oz_ready = false;
  void* oz_a = nullptr;
  cudaStream_t oz_stream = nullptr;
  alignas(64) unsigned char oz_map[8][128] = {};
  // fixed-point digits of a complex128 dense matrix for the integer-pipe
  // sweep (fx.cuh), made on first use: n x n int4 digits (leading dimension
  // n), then n row exponents and a flag word
  int fx_state = 0;   // 0 not made, 1 ready, -1 unusable (non-finite entry, or no memory)
  void* fx_a = nullptr;
  cudaStream_t fx_stream = nullptr;
};

struct ccg_handle {
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  // grow-only device arena holding vectors, partial sums and solve state
  char* arena = nullptr;
  size_t arena_bytes = 0;
  // pinned host poll slots and their events
  void* pinned = nullptr;
  cudaEvent_t poll_ev[2] = {nullptr, nullptr};
  // operator-sweep timing, per ccg_sweep_kind
  bool timing = false;
  std::vector<cudaEvent_t> tev;  // start/stop pairs
  std::vector<int> tev_kind;     // dtype * CCG_SWEEP_KINDS + sweep kind of each pair
  size_t tev_used = 0;
  int* skip_rec = nullptr;       // device, one flag per timed sweep: 1 if it found the solve stopped
  size_t skip_cap = 0;
  int64_t timed_sweeps[2 * CCG_SWEEP_KINDS] = {};
  double timed_ms[2 * CCG_SWEEP_KINDS] = {};
  double bytes_per_sweep[2 * CCG_SWEEP_KINDS] = {};
  // kernels launched by this handle
  int64_t launches = 0;
  // first nonzero return of an operator callback during the current call
  int cb_status = 0;
  // tensor-core block products: enabled flag, staging for split blocks and
  // the pipeline's error flag (first 256 bytes)
  int tc_mode = 1;   // 0 never, 1 refined inner solves and block products, 2 also plain batched solves
  int tc_terms = 2;  // bf16 terms of the split operands (2 or 3; the fp32 accumulation limits both to ~1e-4 at K ~ 1e4)
  int phase_elems = 1;  // floor on the elements per thread of the fused update kernels' grid
  int gm_restart = 30;  // GMRES cycle length m
  int bicgstab_l = 2;   // degree l of BiCGstab(l)
  void* tc_buf = nullptr;
  size_t tc_bytes = 0;
  size_t tc_flag_bytes = 0;   // bytes of the stream-K flags zeroed since the buffer was made
  unsigned tc_epoch = 0;      // launches of the split-bf16 product (the flags' epoch)
  // exact tensor-core block products (integer digit slices; FP64-accurate
  // for complex128, FP32-accurate for complex64): enabled flag, staging for
  // the block's slices and the pipeline's error flag (first 256 bytes)
  int tc_exact = 1;
  void* oz_buf = nullptr;
  size_t oz_bytes = 0;
  // persistent solves (persist.cu): enabled flag, blocks per SM (0: the
  // occupancy limit), the group barriers' wait limit in SM clock cycles, and
  // the test hook that withholds one block's arrival
  int persistent = 2;   // 0 never, 1 always, 2 as the tuned table says (tune_table.h)
  int pk_blocks = 0;
  int fx_mode = 1;   // complex128 A x: 1 fixed-point digits on the integer pipe, 0 the FP64 pipe
  int pdl = 1;       // kernel-per-step loop: programmatic dependent launch of its kernels
  long long wait_limit = 4ll << 30;
  int test_withhold = 0;
  // per timed pair: the units (sweeps) and bytes it stands for
  std::vector<int64_t> tev_units;
  std::vector<double> tev_bytes;
  double timed_bytes[2 * CCG_SWEEP_KINDS] = {};
};

namespace ccg {

// Ensure the arena holds at least `bytes`; synchronises the stream before a
// reallocation.  Returns a ccg_status.
int arena_reserve(ccg_handle* h, size_t bytes);

// Timing hooks around one operator sweep (no-ops unless timing is enabled).
void timing_begin(ccg_handle* h);
void timing_end(ccg_handle* h, int dtype, int kind, double bytes);
void timing_collect(ccg_handle* h);
// The last timed pair stands for `units` sweeps of `bytes` in total (a
// persistent launch); 0 units leaves it out.
void timing_set_units(ccg_handle* h, int64_t units, double bytes);
// Device flag of the sweep being timed (between timing_begin and timing_end),
// or nullptr when timing is off.
int* timing_rec(ccg_handle* h);

// Entry points implemented in solve.cu.
int solve_dense(ccg_handle* h, int method, const ccg_operator* op, const void* y, void* x, double tol, int maxit,
                double* res_hist, ccg_info* info);
int solve_refined(ccg_handle* h, int method, const ccg_operator* op, const ccg_operator* op_in, const void* y,
                  void* x, double tol, int max_outer, double inner_tol, int inner_maxit, double* res_hist,
                  int* inner_iters, ccg_info* info);
int dipole_create(ccg_operator* op, const uint8_t* occ, cudaStream_t s);
void dipole_free(ccg_operator* op);
// y = A x (conj = false) or A^H x (conj = true), enqueued on s; kernels skip
// when st says the solve has stopped (st may be null), and then set
// *skip_rec when it is given (timed sweeps); pdl launches the kernels with
// programmatic dependent launch.
int dipole_apply(const ccg_operator* op, const double2* x, double2* y, bool conj, const SolveState* st,
                 cudaStream_t s, int* skip_rec = nullptr, bool pdl = false);
int dipole_apply(const ccg_operator* op, const float2* x, float2* y, bool conj, const SolveState* st,
                 cudaStream_t s, int* skip_rec = nullptr, bool pdl = false);
int solve_batched(ccg_handle* h, const ccg_operator* op, int64_t k, const void* Y, int64_t ldy, void* X, int64_t ldx,
                  double tol, int maxit, int32_t* iters, int32_t* status, double* relres);
int solve_batched_refined(ccg_handle* h, const ccg_operator* op, const ccg_operator* op_in, int64_t k, const void* Y,
                          int64_t ldy, void* X, int64_t ldx, double tol, int max_outer, double inner_tol,
                          int inner_maxit, int32_t* outer_out, int32_t* inner_out, int32_t* status, double* relres);
bool tc_available(const ccg_operator* op);
int tc_block_product(ccg_handle* h, const ccg_operator* op, const float2* X, float2* Y, int k, const int* skip);
int tc_check_error(ccg_handle* h);
void tc_free(ccg_operator* op);
bool oz_available(const ccg_operator* op);
int oz_block_product(ccg_handle* h, const ccg_operator* op, const double2* X, double2* Y, int k, const int* skip);
int oz_block_product(ccg_handle* h, const ccg_operator* op, const float2* X, float2* Y, int k, const int* skip);
int oz_check_error(ccg_handle* h);
void oz_free(ccg_operator* op);
// The fixed-point digits of a complex128 dense operator (made on first use,
// on the handle's stream); false when the operator cannot use them.
bool fx_prepare(ccg_handle* h, const ccg_operator* op);
void fx_free(ccg_operator* op);
int block_matvec(ccg_handle* h, const ccg_operator* op, int64_t k, const void* X, int64_t ldx, void* Y, int64_t ldy);
// Many dense systems in one persistent launch each (persist.cu).
int solve_multi(ccg_handle* h, int method, int count, const ccg_operator* const* ops, const void* const* y,
                void* const* x, const double* tol, int maxit, int32_t* iters, int32_t* status, double* relres);
int solve_multi_refined(ccg_handle* h, int method, int count, const ccg_operator* const* ops,
                        const ccg_operator* const* ops_in, const void* const* y, void* const* x, const double* tol,
                        int max_outer, double inner_tol, int inner_maxit, int32_t* outer, int32_t* inner,
                        int32_t* status, double* relres);
// Resident blocks of the persistent launch for `method` on complex64 (dtype
// CCG_C64) or complex128 operators: the most systems one launch takes.
int pk_capacity(ccg_handle* h, int method, int dtype);
int matvec_dense(ccg_handle* h, const ccg_operator* op, int trans, const void* x, void* y);
int dot_device(ccg_handle* h, ccg_dtype dtype, int64_t n, const void* u, const void* v, int conj, double* out2);

}  // namespace ccg
