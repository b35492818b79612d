"""numpy-facing wrapper of the C++ CPU oracle (ccg_oracle.cpp).

TEST INFRASTRUCTURE ONLY.  Everything here is a thin marshalling layer:
the arithmetic lives in ccg_oracle.cpp, which restates the textbook methods
the CCGPAK manual names (Sec. 2.1 PIM: BiCGSTAB, CGNR, QMR, BiCG, GMRES(m), CGS,
CGNE, TFQMR; Sec. 3.1 BiCGstab(l); Sec. 2.2
the Sarkar complex-symmetric CG; Sec. 3.4 COCR) and the discrete-dipole
operator of its DDSCAT application (Sec. 1).
"""
import ctypes
import threading

import numpy as np

from . import build as _build

BICGSTAB, CGNR, QMR, COCG, COCR, BICG, GMRES, CGS, CGNE, TFQMR, BICGSTABL = range(11)
METHODS = {"bicgstab": BICGSTAB, "cgnr": CGNR, "qmr": QMR, "cocg": COCG, "cocr": COCR, "bicg": BICG,
           "gmres": GMRES, "cgs": CGS, "cgne": CGNE, "tfqmr": TFQMR, "bicgstabl": BICGSTABL}
OK, NOT_CONVERGED, BREAKDOWN, INVALID = 0, 1, 2, -1

_libs = {}
_lock = threading.Lock()


def lib(parallel=False):
    """The serial oracle library, or with parallel=True its OpenMP build
    (same source; the dense products' independent output elements on all
    allowed host cores, bit-identical results)."""
    with _lock:
        if parallel not in _libs:
            path = _build.build_omp() if parallel else _build.build()
            L = ctypes.CDLL(path)
            vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            L.orc_abi_version.restype = i32
            L.orc_threads.restype = i32
            L.orc_op_dense_c128.restype = vp
            L.orc_op_dense_c128.argtypes = [i64, i64, vp, i32]
            L.orc_op_dense_c64.restype = vp
            L.orc_op_dense_c64.argtypes = [i64, i64, vp, i32]
            L.orc_op_dipole.restype = vp
            L.orc_op_dipole.argtypes = [i32, i32, i32, vp, dbl, dbl, dbl, i32]
            L.orc_op_destroy.argtypes = [vp]
            L.orc_op_n.restype = i64
            L.orc_op_n.argtypes = [vp]
            L.orc_dipole_nsites.restype = i64
            L.orc_dipole_nsites.argtypes = [vp]
            L.orc_dipole_alpha.argtypes = [vp, vp]
            L.orc_dipole_sites.argtypes = [vp, vp]
            L.orc_dipole_rows.argtypes = [vp, vp, vp, i64, vp]
            L.orc_green.argtypes = [dbl, dbl, dbl, dbl, vp]
            L.orc_matvec_c128.argtypes = [vp, i32, vp, vp]
            L.orc_matvec_c64.argtypes = [vp, i32, vp, vp]
            L.orc_solve_c128.argtypes = [vp, i32, vp, vp, dbl, i32, vp, vp, vp]
            L.orc_solve_c64.argtypes = [vp, i32, vp, vp, dbl, i32, vp, vp, vp]
            L.orc_refine.argtypes = [vp, vp, i32, vp, vp, dbl, i32, dbl, i32, vp, vp]
            L.orc_fft3d.argtypes = [vp, i64, i64, i64, i32]
            L.orc_set_restart.argtypes = [i32]
            L.orc_set_bicgstab_l.argtypes = [i32]
            _libs[parallel] = L
    return _libs[parallel]


def threads(parallel=False):
    """Host threads the dense products of that build use."""
    return int(lib(parallel).orc_threads())


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


class _Op:
    """Owns an oracle operator handle and the arrays it points into."""

    def __init__(self, handle, n, dtype, keep=(), L=None):
        self.h = handle
        self.n = int(n)
        self.dtype = np.dtype(dtype)
        self._keep = keep
        self.L = lib() if L is None else L   # the library that owns the handle

    def __del__(self):
        if getattr(self, "h", None):
            self.L.orc_op_destroy(self.h)
            self.h = None

    def matvec(self, x, trans=False):
        """A x (trans=False) or A^H x (trans=True)."""
        x = np.ascontiguousarray(x, dtype=self.dtype)
        y = np.empty(self.n, dtype=self.dtype)
        fn = self.L.orc_matvec_c128 if self.dtype == np.complex128 else self.L.orc_matvec_c64
        fn(self.h, int(bool(trans)), _ptr(x), _ptr(y))
        return y


class DenseOp(_Op):
    """Dense row-major complex matrix (complex128 or complex64).

    symmetric=True marks A = A^T (verified here exactly), which COCG needs.
    parallel=True applies it with the OpenMP build (same results).
    """

    def __init__(self, A, symmetric=False, parallel=False):
        A = np.ascontiguousarray(A)
        assert A.ndim == 2 and A.shape[0] == A.shape[1]
        assert A.dtype in (np.complex128, np.complex64)
        if symmetric:
            assert np.array_equal(A, A.T), "matrix is not complex symmetric"
        n = A.shape[0]
        L = lib(parallel)
        fn = L.orc_op_dense_c128 if A.dtype == np.complex128 else L.orc_op_dense_c64
        super().__init__(fn(n, n, _ptr(A), int(bool(symmetric))), n, A.dtype, keep=(A,), L=L)


class DipoleOp(_Op):
    """Discrete-dipole operator on the occupied sites of an nx*ny*nz lattice.

    occ is a uint8 array of shape (nx, ny, nz).  Unknowns are ordered
    v[a*N + s] (component a in x, y, z; site s lexicographic with the last
    axis fastest).  use_fft selects the circulant FFT form of the same sum.
    Arithmetic is in double; dtype=complex64 rounds inputs and results.
    """

    def __init__(self, occ, kd, m, use_fft=False, dtype=np.complex128):
        occ = np.ascontiguousarray(occ, dtype=np.uint8)
        assert occ.ndim == 3
        nx, ny, nz = occ.shape
        m = complex(m)
        h = lib().orc_op_dipole(nx, ny, nz, _ptr(occ), float(kd), m.real, m.imag, int(bool(use_fft)))
        self.nsites = int(lib().orc_dipole_nsites(h))
        super().__init__(h, 3 * self.nsites, dtype, keep=(occ,))

    @property
    def alpha(self):
        out = np.zeros(2)
        lib().orc_dipole_alpha(self.h, _ptr(out))
        return complex(out[0], out[1])

    def sites(self):
        out = np.zeros((self.nsites, 3), dtype=np.int32)
        lib().orc_dipole_sites(self.h, _ptr(out))
        return out

    def rows(self, x, sel=None):
        """Direct-sum (A x) at the listed sites; returns shape (3, len(sel))."""
        x = np.ascontiguousarray(x, dtype=np.complex128)
        if sel is None:
            sel_arr, nsel, sp = None, self.nsites, ctypes.c_void_p(0)
        else:
            sel_arr = np.ascontiguousarray(sel, dtype=np.int64)
            nsel, sp = len(sel_arr), _ptr(sel_arr)
        y = np.empty(3 * nsel, dtype=np.complex128)
        lib().orc_dipole_rows(self.h, _ptr(x), _ptr(y), nsel, sp)
        return y.reshape(3, nsel)


class _View(_Op):
    def __init__(self, owner, dtype):
        self.h = owner.h
        self.n = owner.n
        self.dtype = np.dtype(dtype)
        self.L = owner.L
        self._owner = owner

    def __del__(self):
        pass


def view(op, dtype):
    """The same oracle operator used at another working precision (dipole only)."""
    return _View(op, dtype)


class SolveResult:
    def __init__(self, x, iters, status, detail, hist, tau=None):
        self.x, self.iters, self.status, self.detail = x, iters, status, detail
        self.hist = hist
        self.tau = tau

    def __repr__(self):
        return "SolveResult(iters=%d, status=%d, detail=%d, relres=%.3e)" % (
            self.iters, self.status, self.detail, self.hist[-1] if len(self.hist) else float("nan"))


def solve(op, method, y, x0=None, tol=1e-10, maxit=1000, want_tau=False, restart=30, ell=2):
    """Run one oracle method; returns SolveResult with hist[k] = ||r_k||/||y||
    (restart: the cycle length m of GMRES(m); ell: the degree of BiCGstab(l))."""
    m = METHODS[method] if isinstance(method, str) else int(method)
    L = op.L
    L.orc_set_restart(int(restart))
    L.orc_set_bicgstab_l(int(ell))
    y = np.ascontiguousarray(y, dtype=op.dtype)
    x = np.zeros(op.n, dtype=op.dtype) if x0 is None else np.array(x0, dtype=op.dtype, copy=True)
    hist = np.full(maxit + 1, np.nan)
    tau = np.full(maxit + 1, np.nan) if want_tau else None
    out = np.zeros(3, dtype=np.int32)
    fn = L.orc_solve_c128 if op.dtype == np.complex128 else L.orc_solve_c64
    fn(op.h, m, _ptr(y), _ptr(x), float(tol), int(maxit), _ptr(out), _ptr(hist),
       _ptr(tau) if want_tau else ctypes.c_void_p(0))
    it = int(out[0])
    return SolveResult(x, it, int(out[1]), int(out[2]), hist[: it + 1], None if tau is None else tau[: it + 1])


def refine(op64, op32, method, y, x0=None, tol=1e-10, max_outer=20, inner_tol=1e-4, inner_maxit=50, restart=30,
           ell=2):
    """FP64 iterative refinement around an FP32 inner solve.

    Returns (x, outer_steps, status, inner_iterations, hist_outer).
    """
    m = METHODS[method] if isinstance(method, str) else int(method)
    L = op64.L
    assert op32.L is L, "both operators must come from the same oracle build"
    L.orc_set_restart(int(restart))
    L.orc_set_bicgstab_l(int(ell))
    y = np.ascontiguousarray(y, dtype=np.complex128)
    x = np.zeros(op64.n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128, copy=True)
    hist = np.full(max_outer + 1, np.nan)
    out = np.zeros(4, dtype=np.int32)
    L.orc_refine(op64.h, op32.h, m, _ptr(y), _ptr(x), float(tol), int(max_outer), float(inner_tol),
                     int(inner_maxit), _ptr(out), _ptr(hist))
    return x, int(out[0]), int(out[1]), int(out[3]), hist[: int(out[0]) + 1]


def green(kd, r):
    """Field tensor G(r) (3x3 complex) of a unit dipole at displacement r."""
    out = np.zeros(12)
    lib().orc_green(float(kd), float(r[0]), float(r[1]), float(r[2]), _ptr(out))
    c = out[0::2] + 1j * out[1::2]
    xx, xy, xz, yy, yz, zz = c
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def fft3d(g, sign=-1):
    """Unnormalised 3D DFT with exp(sign*2*pi*i*jk/n) kernels."""
    g = np.array(g, dtype=np.complex128, copy=True, order="C")
    assert g.ndim == 3
    lib().orc_fft3d(_ptr(g), g.shape[0], g.shape[1], g.shape[2], int(sign))
    return g
