"""Python binding of libccg (include/ccg.h): argument marshalling only.

Every computation runs in libccg.so's CUDA kernels; this module only turns
torch tensors / numpy arrays into pointers and sizes.  There is no CPU
fallback: if libccg.so is missing or no CUDA device is present, calls raise.

Device memory and streams come from PyTorch: pass CUDA tensors (complex128
or complex64) and, optionally, a torch.cuda.Stream.  ccg_solve also takes
numpy arrays (host memory), which the library copies through its own
workspace.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libccg.so")

BICGSTAB, CGNR, QMR, COCG, COCR, BICG, GMRES, CGS, CGNE, TFQMR, BICGSTABL = range(11)
METHODS = {"bicgstab": BICGSTAB, "cgnr": CGNR, "qmr": QMR, "cocg": COCG, "cocr": COCR, "bicg": BICG,
           "gmres": GMRES, "cgs": CGS, "cgne": CGNE, "tfqmr": TFQMR, "bicgstabl": BICGSTABL}
C64, C128 = 0, 1
OK, NOT_CONVERGED, BREAKDOWN = 0, 1, 2
ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
OP_SYMMETRIC = 1
OPT_TENSOR_CORES = 1
OPT_TC_SPLIT = 2
OPT_GMRES_RESTART = 3
OPT_BICGSTAB_L = 4
OPT_TC_EXACT = 5
OPT_PERSISTENT = 6
OPT_PK_BLOCKS = 7
OPT_WAIT_LIMIT = 8
OPT_TEST_WITHHOLD = 9
OPT_FP64_SWEEP = 10
OPT_PDL = 11

PIPE_FP64_FMA = 0
PIPE_FP32_FMA = 1
PIPE_IMAD_WIDE = 2
PIPE_MAD_WIDE_PTX = 3
PIPE_MAD_PAIR_PTX = 4

# ccg_matvec_fn: int (*)(void* ctx, int64_t n, const void* x, void* y, void* stream)
MATVEC_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_void_p)
SWEEP_N, SWEEP_C, SWEEP_BOTH, SWEEP_BLOCK, SWEEP_BLOCK_TC, SWEEP_BLOCK_EXACT, SWEEP_PERSIST = 0, 1, 2, 3, 4, 5, 6

_lib = None


class CcgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libccg status %d: %s" % (status, msg))
        self.status = status


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("breakdown", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("relres", ctypes.c_double), ("true_relres", ctypes.c_double),
                ("ynorm", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nrhs", ctypes.c_int32), ("n", ctypes.c_int64), ("shift", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("L", ctypes.c_int32), ("maxit", ctypes.c_int32), ("kd", ctypes.c_double),
                ("m_re", ctypes.c_double), ("m_im", ctypes.c_double), ("tol", ctypes.c_double),
                ("keep_x", ctypes.c_int32), ("mode", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("relres", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("n", ctypes.c_int64), ("nrhs", ctypes.c_int32), ("slot", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


REQ_DENSE, REQ_DIPOLE = 0, 1


def lib():
    """Load libccg.so (built by paper_1208_4869_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libccg.so is not built (%s); run paper_1208_4869_gb300.build.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.ccg_abi_version.restype = i32
    L.ccg_last_error.restype = ctypes.c_char_p
    L.ccg_status_string.restype = ctypes.c_char_p
    L.ccg_status_string.argtypes = [i32]
    L.ccg_create.argtypes = [ctypes.POINTER(vp), vp]
    L.ccg_destroy.argtypes = [vp]
    L.ccg_set_stream.argtypes = [vp, vp]
    L.ccg_op_dense.argtypes = [vp, i32, i64, vp, i64, i32, ctypes.POINTER(vp)]
    L.ccg_op_destroy.argtypes = [vp]
    L.ccg_op_dipole.argtypes = [vp, i32, i32, i32, i32, vp, dbl, dbl, dbl, ctypes.POINTER(vp)]
    L.ccg_op_callback.argtypes = [vp, i32, i64, MATVEC_FN, MATVEC_FN, vp, i32, ctypes.POINTER(vp)]
    L.ccg_dipole_sites.restype = i64
    L.ccg_dipole_sites.argtypes = [vp]
    L.ccg_op_size.restype = i64
    L.ccg_op_size.argtypes = [vp]
    L.ccg_matvec.argtypes = [vp, vp, i32, vp, vp]
    L.ccg_dot.argtypes = [vp, i32, i64, vp, vp, i32, vp]
    L.ccg_solve.argtypes = [vp, i32, vp, vp, vp, dbl, i32, vp, ctypes.POINTER(Info)]
    L.ccg_timing_enable.argtypes = [vp, i32]
    L.ccg_timing_read.argtypes = [vp, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    L.ccg_solve_refined.argtypes = [vp, i32, vp, vp, vp, vp, dbl, i32, dbl, i32, vp, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(Info)]
    L.ccg_timing_reset.argtypes = [vp]
    L.ccg_solve_batched.argtypes = [vp, i32, vp, i64, vp, i64, vp, i64, dbl, i32, vp, vp, vp]
    L.ccg_solve_batched_refined.argtypes = [vp, i32, vp, vp, i64, vp, i64, vp, i64, dbl, i32, dbl, i32, vp, vp, vp, vp]
    L.ccg_block_matvec.argtypes = [vp, vp, i64, vp, i64, vp, i64]
    L.ccg_set_option.argtypes = [vp, i32, i32]
    L.ccg_solve_multi.argtypes = [vp, i32, i64, vp, vp, vp, vp, i32, vp, vp, vp]
    L.ccg_solve_multi_refined.argtypes = [vp, i32, i64, vp, vp, vp, vp, vp, i32, dbl, i32, vp, vp, vp, vp]
    L.ccg_server_create.argtypes = [ctypes.POINTER(vp), i32, i32, ctypes.c_uint64]
    L.ccg_server_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(i64)]
    L.ccg_server_poll.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int)]
    L.ccg_server_wait.argtypes = [vp, i64, ctypes.POINTER(Result), vp]
    L.ccg_server_now.restype = dbl
    L.ccg_server_now.argtypes = [vp]
    L.ccg_server_estimate.argtypes = [ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.ccg_server_charged.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    L.ccg_server_set_batching.argtypes = [vp, i64, i32]
    L.ccg_server_destroy.argtypes = [vp]
    L.ccg_launch_count.restype = i64
    L.ccg_launch_count.argtypes = [vp]
    L.ccg_pipe_rate.restype = i32
    L.ccg_pipe_rate.argtypes = [vp, i32, ctypes.POINTER(dbl)]
    L.ccg_check_block_schedule.restype = i32
    L.ccg_check_block_schedule.argtypes = [i64, i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i64)]
    for name in ("ccg_create", "ccg_destroy", "ccg_set_stream", "ccg_op_dense", "ccg_op_dipole", "ccg_op_destroy", "ccg_matvec",
                 "ccg_dot", "ccg_solve", "ccg_solve_refined", "ccg_solve_batched", "ccg_solve_batched_refined",
                 "ccg_block_matvec", "ccg_set_option", "ccg_solve_multi", "ccg_solve_multi_refined", "ccg_server_create", "ccg_server_submit", "ccg_server_poll",
                 "ccg_server_wait", "ccg_server_destroy", "ccg_server_estimate", "ccg_server_charged", "ccg_server_set_batching",
                 "ccg_timing_enable", "ccg_timing_read", "ccg_timing_reset"):
        getattr(L, name).restype = i32
    if L.ccg_abi_version() != 1:
        raise ImportError("libccg ABI version mismatch")
    _lib = L
    return L


def _check(st):
    if st < 0:
        raise CcgError(st, lib().ccg_last_error().decode())
    return st


def _dtype_code(dt):
    s = str(dt)
    if "complex128" in s:
        return C128
    if "complex64" in s:
        return C64
    raise TypeError("complex64 or complex128 expected, got %s" % s)


def _ptr(a):
    """Pointer of a torch tensor (device or host) or numpy array; must be contiguous."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous or a.ndim == 1
        return ctypes.c_void_p(a.ctypes.data)
    assert a.is_contiguous(), "contiguous tensor expected"
    return ctypes.c_void_p(a.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream) or 0)


class Handle:
    """ccg_create / ccg_destroy: a handle bound to a CUDA stream."""

    def __init__(self, stream=None):
        h = ctypes.c_void_p()
        _check(lib().ccg_create(ctypes.byref(h), _stream_ptr(stream)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().ccg_destroy(self.h)
            self.h = ctypes.c_void_p()

    __del__ = close

    def set_stream(self, stream):
        _check(lib().ccg_set_stream(self.h, _stream_ptr(stream)))

    def op_callback(self, n, dtype, matvec, cmatvec=None, symmetric=False):
        """ccg_op_callback: an operator given by Python callables matvec(x_ptr, y_ptr, stream_ptr) and,
        optionally, cmatvec(...) that enqueue y = A x (resp. A^H x) for device vectors of n complex
        values on the given CUDA stream and return 0 (the manual's matvec / cmatvec)."""
        def wrap(f):
            if f is None:
                return MATVEC_FN()
            def fn(ctx, nn, x, y, stream):
                try:
                    return int(f(x or 0, y or 0, stream or 0) or 0)
                except Exception:  # an exception cannot cross the C boundary: report failure
                    return 1
            return MATVEC_FN(fn)
        code = _dtype_code(dtype)
        fns = (wrap(matvec), wrap(cmatvec))
        op = ctypes.c_void_p()
        _check(lib().ccg_op_callback(self.h, code, int(n), fns[0], fns[1], None,
                                     OP_SYMMETRIC if symmetric else 0, ctypes.byref(op)))
        return Operator(op, fns, code)

    def op_dense(self, A, symmetric=False):
        """ccg_op_dense on a CUDA tensor A (n x n, row-major, complex64/128; rows may be
        padded: a view with stride(1) == 1 and stride(0) = lda >= n); A is not copied."""
        assert A.dim() == 2 and A.shape[0] == A.shape[1] and A.is_cuda
        assert A.stride(1) == 1 and A.stride(0) >= A.shape[1]
        op = ctypes.c_void_p()
        _check(lib().ccg_op_dense(self.h, _dtype_code(A.dtype), A.shape[0], ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                  OP_SYMMETRIC if symmetric else 0, ctypes.byref(op)))
        return Operator(op, A, _dtype_code(A.dtype))

    def op_dipole(self, occ, kd, m, dtype="complex128"):
        """ccg_op_dipole on a host uint8 occupancy array of shape (nx, ny, nz)."""
        occ = np.ascontiguousarray(occ, dtype=np.uint8)
        assert occ.ndim == 3
        code = C128 if "128" in str(dtype) else C64
        op = ctypes.c_void_p()
        m = complex(m)
        _check(lib().ccg_op_dipole(self.h, code, occ.shape[0], occ.shape[1], occ.shape[2],
                                   ctypes.c_void_p(occ.ctypes.data), float(kd), m.real, m.imag, ctypes.byref(op)))
        o = Operator(op, None, code)
        o.nsites = int(lib().ccg_dipole_sites(op))
        return o

    def matvec(self, op, x, y, trans=False):
        """ccg_matvec: y = A x (trans=False) or A^H x (trans=True), device vectors."""
        _check(lib().ccg_matvec(self.h, op.op, int(bool(trans)), _ptr(x), _ptr(y)))
        return y

    def dot(self, u, v, conj=True):
        """ccg_dot: <u, v> (conj) or [u, v] of two device vectors, as a Python complex."""
        out = np.zeros(2)
        _check(lib().ccg_dot(self.h, _dtype_code(u.dtype), u.numel(), _ptr(u), _ptr(v), int(bool(conj)),
                             ctypes.c_void_p(out.ctypes.data)))
        return complex(out[0], out[1])

    def solve(self, method, op, y, x, tol=1e-10, maxit=1000, want_hist=True, want_info=True):
        """ccg_solve.  x holds x0 and receives the solution.  Returns (status, info dict, hist)."""
        m = METHODS[method] if isinstance(method, str) else int(method)
        hist = np.full(maxit + 1, np.nan) if want_hist else None
        info = Info()
        st = lib().ccg_solve(self.h, m, op.op, _ptr(y), _ptr(x), float(tol), int(maxit),
                             ctypes.c_void_p(hist.ctypes.data) if want_hist else ctypes.c_void_p(0),
                             ctypes.byref(info) if want_info else None)
        _check(st)
        d = info.as_dict() if want_info else {}
        if want_hist and want_info:
            hist = hist[: info.iters + 1]
        return st, d, hist

    def solve_refined(self, method, op, op_inner, y, x, tol=1e-10, max_outer=30, inner_tol=1e-5, inner_maxit=200,
                      want_hist=True):
        """ccg_solve_refined: complex128 residual/update around complex64 inner solves.
        Returns (status, info dict, outer residual history, total inner iterations)."""
        m = METHODS[method] if isinstance(method, str) else int(method)
        hist = np.full(max_outer + 1, np.nan) if want_hist else None
        info = Info()
        inner = ctypes.c_int(0)
        st = lib().ccg_solve_refined(self.h, m, op.op, op_inner.op, _ptr(y), _ptr(x), float(tol), int(max_outer),
                                     float(inner_tol), int(inner_maxit),
                                     ctypes.c_void_p(hist.ctypes.data) if want_hist else ctypes.c_void_p(0),
                                     ctypes.byref(inner), ctypes.byref(info))
        _check(st)
        if want_hist:
            hist = hist[: info.iters + 1]
        return st, info.as_dict(), hist, inner.value

    def _block_args(self, op, Y, X):
        n = op.n
        assert Y.dim() == 2 and X.dim() == 2 and Y.shape == X.shape and Y.shape[0] == n
        # column-major blocks: torch tensors of shape (n, k) with stride (1, ld)
        assert Y.stride(0) == 1 and X.stride(0) == 1, "blocks must be column-major (stride (1, ld))"
        return Y.shape[1], ctypes.c_void_p(Y.data_ptr()), max(Y.stride(1), n), ctypes.c_void_p(X.data_ptr()), \
            max(X.stride(1), n)

    def block_matvec(self, op, X, Y):
        """ccg_block_matvec: Y = A X for column-major device blocks of shape (n, k)."""
        k, xp, ldx, yp, ldy = self._block_args(op, X, Y)
        _check(lib().ccg_block_matvec(self.h, op.op, k, xp, ldx, yp, ldy))
        return Y

    def set_option(self, option, value):
        _check(lib().ccg_set_option(self.h, int(option), int(value)))

    def solve_batched(self, method, op, Y, X, tol=1e-10, maxit=1000):
        """ccg_solve_batched on column-major device blocks Y, X of shape (n, k).
        Returns (status, iters, per-column statuses, relres)."""
        k, yp, ldy, xp, ldx = self._block_args(op, Y, X)
        it = np.zeros(k, np.int32)
        sts = np.zeros(k, np.int32)
        rr = np.zeros(k)
        m = METHODS[method] if isinstance(method, str) else int(method)
        st = lib().ccg_solve_batched(self.h, m, op.op, k, yp, ldy, xp, ldx, float(tol), int(maxit),
                                     ctypes.c_void_p(it.ctypes.data), ctypes.c_void_p(sts.ctypes.data),
                                     ctypes.c_void_p(rr.ctypes.data))
        _check(st)
        return st, it, sts, rr

    def solve_batched_refined(self, method, op, op_inner, Y, X, tol=1e-10, max_outer=30, inner_tol=1e-5,
                              inner_maxit=200):
        """ccg_solve_batched_refined.  Returns (status, outer, inner, per-column statuses, relres)."""
        k, yp, ldy, xp, ldx = self._block_args(op, Y, X)
        outer = np.zeros(k, np.int32)
        inner = np.zeros(k, np.int32)
        sts = np.zeros(k, np.int32)
        rr = np.zeros(k)
        m = METHODS[method] if isinstance(method, str) else int(method)
        st = lib().ccg_solve_batched_refined(self.h, m, op.op, op_inner.op, k, yp, ldy, xp, ldx, float(tol),
                                             int(max_outer), float(inner_tol), int(inner_maxit),
                                             ctypes.c_void_p(outer.ctypes.data), ctypes.c_void_p(inner.ctypes.data),
                                             ctypes.c_void_p(sts.ctypes.data), ctypes.c_void_p(rr.ctypes.data))
        _check(st)
        return st, outer, inner, sts, rr

    @staticmethod
    def _ptr_array(items):
        arr = (ctypes.c_void_p * len(items))()
        for i, it in enumerate(items):
            arr[i] = it if isinstance(it, int) else (it.op.value if isinstance(it, Operator) else _ptr(it).value)
        return arr

    def solve_multi(self, method, ops, ys, xs, tol=1e-10, maxit=1000):
        """ccg_solve_multi: many dense systems in one launch.  ops, ys, xs are lists
        (xs: start vectors in, solutions out).  Returns (status, iters, statuses, relres)."""
        k = len(ops)
        m = METHODS[method] if isinstance(method, str) else int(method)
        tols = np.ascontiguousarray(np.broadcast_to(np.asarray(tol, dtype=np.float64), (k,)))
        iters = np.zeros(k, np.int32)
        sts = np.zeros(k, np.int32)
        rr = np.zeros(k)
        st = lib().ccg_solve_multi(self.h, m, k, self._ptr_array(ops), self._ptr_array(ys), self._ptr_array(xs),
                                   ctypes.c_void_p(tols.ctypes.data), int(maxit), ctypes.c_void_p(iters.ctypes.data),
                                   ctypes.c_void_p(sts.ctypes.data), ctypes.c_void_p(rr.ctypes.data))
        _check(st)
        return st, iters, sts, rr

    def solve_multi_refined(self, method, ops, ops_inner, ys, xs, tol=1e-10, max_outer=30, inner_tol=1e-5,
                            inner_maxit=200):
        """ccg_solve_multi_refined.  Returns (status, outer, inner, statuses, relres)."""
        k = len(ops)
        m = METHODS[method] if isinstance(method, str) else int(method)
        tols = np.ascontiguousarray(np.broadcast_to(np.asarray(tol, dtype=np.float64), (k,)))
        outer = np.zeros(k, np.int32)
        inner = np.zeros(k, np.int32)
        sts = np.zeros(k, np.int32)
        rr = np.zeros(k)
        st = lib().ccg_solve_multi_refined(self.h, m, k, self._ptr_array(ops), self._ptr_array(ops_inner),
                                           self._ptr_array(ys), self._ptr_array(xs), ctypes.c_void_p(tols.ctypes.data),
                                           int(max_outer), float(inner_tol), int(inner_maxit),
                                           ctypes.c_void_p(outer.ctypes.data), ctypes.c_void_p(inner.ctypes.data),
                                           ctypes.c_void_p(sts.ctypes.data), ctypes.c_void_p(rr.ctypes.data))
        _check(st)
        return st, outer, inner, sts, rr

    def timing(self, enable=None, reset=False, kind=SWEEP_N, dtype=C128):
        """Per-sweep CUDA-event timing of one precision and sweep kind: (sweeps, total_ms, bytes_per_sweep)."""
        if enable is not None:
            _check(lib().ccg_timing_enable(self.h, int(bool(enable))))
        if reset:
            _check(lib().ccg_timing_reset(self.h))
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        b = ctypes.c_double()
        _check(lib().ccg_timing_read(self.h, int(dtype), int(kind), ctypes.byref(n), ctypes.byref(ms),
                                     ctypes.byref(b)))
        return n.value, ms.value, b.value

    def launch_count(self):
        """ccg_launch_count: kernels this handle has launched."""
        return int(lib().ccg_launch_count(self.h))

    def pipe_rate(self, pipe):
        """ccg_pipe_rate: measured Gop/s of an arithmetic pipe (PIPE_FP64_FMA,
        PIPE_FP32_FMA, PIPE_IMAD_WIDE)."""
        out = ctypes.c_double()
        _check(lib().ccg_pipe_rate(self.h, pipe, ctypes.byref(out)))
        return out.value


class Operator:
    def __init__(self, op, keep, dtype_code):
        self.op = op
        self._keep = keep
        self.dtype_code = dtype_code

    @property
    def n(self):
        return int(lib().ccg_op_size(self.op))

    def close(self):
        if getattr(self, "op", None) and self.op.value:
            lib().ccg_op_destroy(self.op)
            self.op = ctypes.c_void_p()

    __del__ = close


def make_request(kind="dense", n=0, nrhs=1, shift=3.0, seed=0, L=0, kd=0.5, m=1.5 + 0.01j, tol=1e-10, maxit=0,
                 keep_x=False, mode=0):
    r = Request()
    r.kind = REQ_DENSE if kind == "dense" else REQ_DIPOLE
    r.n, r.nrhs, r.shift, r.seed, r.L, r.maxit = int(n), int(nrhs), float(shift), int(seed), int(L), int(maxit)
    r.kd, r.m_re, r.m_im, r.tol, r.keep_x = float(kd), complex(m).real, complex(m).imag, float(tol), int(keep_x)
    r.mode = int(mode)
    return r


def check_block_schedule(n, k, terms, sms):
    """ccg_check_block_schedule: (CTAs of the launch, violations found) of the
    tensor-core block product's work split, checked on the host."""
    ctas, bad = ctypes.c_int(), ctypes.c_int64()
    _check(lib().ccg_check_block_schedule(n, k, terms, sms, ctypes.byref(ctas), ctypes.byref(bad)))
    return ctas.value, bad.value


def server_estimate(**req):
    """ccg_server_estimate: device bytes the serving admission charges for a request."""
    b = ctypes.c_uint64()
    _check(lib().ccg_server_estimate(ctypes.byref(make_request(**req)), ctypes.byref(b)))
    return b.value


class Server:
    """ccg_server_*: a queue of solve requests served by `slots` workers on one
    GPU under an HBM budget (bytes; 0 = 120 GB)."""

    def __init__(self, device=0, slots=4, budget_bytes=0):
        sv = ctypes.c_void_p()
        _check(lib().ccg_server_create(ctypes.byref(sv), int(device), int(slots), int(budget_bytes)))
        self.sv = sv
        self._sizes = {}

    def submit(self, kind="dense", n=0, nrhs=1, shift=3.0, seed=0, L=0, kd=0.5, m=1.5 + 0.01j, tol=1e-10,
               maxit=0, keep_x=False, mode=0):
        r = make_request(kind, n, nrhs, shift, seed, L, kd, m, tol, maxit, keep_x, mode)
        t = ctypes.c_int64()
        _check(lib().ccg_server_submit(self.sv, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        d = ctypes.c_int()
        _check(lib().ccg_server_poll(self.sv, int(ticket), ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket, x_size=0):
        """Result dict, and the solution (complex128, column-major n x nrhs) if x_size > 0."""
        res = Result()
        x = np.zeros(x_size, np.complex128) if x_size else None
        _check(lib().ccg_server_wait(self.sv, int(ticket), ctypes.byref(res),
                                     ctypes.c_void_p(x.ctypes.data) if x_size else ctypes.c_void_p(0)))
        return res.as_dict(), x

    def now(self):
        return lib().ccg_server_now(self.sv)

    def set_batching(self, max_n=2048, max_systems=256):
        """ccg_server_set_batching: small dense requests solved together (max_n = 0: off)."""
        _check(lib().ccg_server_set_batching(self.sv, int(max_n), int(max_systems)))

    def charged(self):
        """ccg_server_charged: bytes charged against the budget now."""
        b = ctypes.c_uint64()
        _check(lib().ccg_server_charged(self.sv, ctypes.byref(b)))
        return b.value

    def close(self):
        if getattr(self, "sv", None) and self.sv.value:
            lib().ccg_server_destroy(self.sv)
            self.sv = ctypes.c_void_p()

    __del__ = close
