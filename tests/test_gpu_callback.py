"""User-supplied operators through the C ABI: the manual's `matvec` and
`cmatvec` (Sec. 5) as host callbacks that enqueue the product on the solve's
stream (ccg_op_callback).

The callbacks here apply a built-in operator through a second handle bound
to the same stream, so a solve through the callback operator runs the same
products as a solve through the built-in one: iterates agree to 1e-12 in
complex128 (QMR and BiCG within 1e-9: the built-in dense operator forms
A p and A^H q in one fused sweep whose partial sums are added in another
order) and with the CPU oracle as in the dense parity tests.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1208_4869_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ccg():
    from paper_1208_4869_gb300 import build as B
    B.build()
    from paper_1208_4869_gb300 import ccg as C
    return C


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


class Wrapped:
    """Callbacks that apply `inner` (a built-in operator) with handle `h2`,
    bound to whatever stream the solve passes in.  Counts the calls."""

    def __init__(self, ccg, h2, inner, fail_after=None):
        self.ccg, self.h2, self.inner = ccg, h2, inner
        self.calls = 0
        self.fail_after = fail_after

    def _apply(self, trans, x, y, stream):
        self.calls += 1
        if self.fail_after is not None and self.calls > self.fail_after:
            return 7
        L = self.ccg.lib()
        if L.ccg_set_stream(self.h2.h, ctypes.c_void_p(stream)) != 0:
            return 1
        return L.ccg_matvec(self.h2.h, self.inner.op, trans, ctypes.c_void_p(x), ctypes.c_void_p(y))

    def matvec(self, x, y, stream):
        return self._apply(0, x, y, stream)

    def cmatvec(self, x, y, stream):
        return self._apply(1, x, y, stream)


def callback_op(ccg, h, h2, inner, n, dtype, symmetric=False, with_c=True, fail_after=None):
    w = Wrapped(ccg, h2, inner, fail_after)
    op = h.op_callback(n, dtype, w.matvec, w.cmatvec if with_c else None, symmetric=symmetric)
    return op, w


@pytest.mark.parametrize("method", ["bicgstab", "cgnr", "qmr", "cocg", "cocr", "bicg", "gmres", "cgs", "cgne",
                                    "tfqmr", "bicgstabl"])
def test_callback_dense_matches_builtin(ccg, method):
    n = 256
    sym = method in ("cocg", "cocr")

    def system(shift, seed):
        A, y = W.dense_system(n, shift, seed)
        return ((A + A.T) / 2 if sym else A), y

    A, y = system(0.6, 5)                  # slow enough to run 12 iterations
    h, h2 = ccg.Handle(), ccg.Handle()
    opd = h2.op_dense(dev(A), symmetric=sym)
    opc, w = callback_op(ccg, h, h2, opd, n, "complex128", symmetric=sym)
    opb = h.op_dense(dev(A), symmetric=sym)
    oop = O.DenseOp(A, symmetric=sym)
    for it in (3, 12):
        xs = []
        for op in (opc, opb):
            x = dev(np.zeros(n, np.complex128))
            h.solve(method, op, dev(y), x, tol=0.0, maxit=it)
            xs.append(x.cpu().numpy())
        ref = O.solve(oop, method, y, tol=0.0, maxit=it)
        tol = 1e-9 if method in ("qmr", "bicg") else 1e-12
        assert relerr(xs[0], xs[1]) < tol, (method, it, relerr(xs[0], xs[1]))
        assert relerr(xs[0], ref.x) < 1e-9, (method, it)
    assert w.calls > 0
    # a converged solve on a well-conditioned system, and its true residual
    A, y = system(3.0, 1)
    opd = h2.op_dense(dev(A), symmetric=sym)
    opc, _ = callback_op(ccg, h, h2, opd, n, "complex128", symmetric=sym)
    x = dev(np.zeros(n, np.complex128))
    st, info, hist = h.solve(method, opc, dev(y), x, tol=1e-10, maxit=1000)
    assert st == 0 and info["true_relres"] <= 1e-9
    xh = x.cpu().numpy()
    assert np.linalg.norm(y - A @ xh) / np.linalg.norm(y) <= 1e-9


def test_callback_matvec_api(ccg):
    n = 257
    A, _ = W.dense_system(n, 1.0, 5)
    xv = W.random_vector(n, 6)
    h, h2 = ccg.Handle(), ccg.Handle()
    opd = h2.op_dense(dev(A))
    opc, _ = callback_op(ccg, h, h2, opd, n, "complex128")
    for trans in (False, True):
        y = dev(np.zeros(n, np.complex128))
        h.matvec(opc, dev(xv), y, trans=trans)
        torch.cuda.synchronize()
        ref = (A.conj().T if trans else A) @ xv
        assert relerr(y.cpu().numpy(), ref) < 1e-13


def test_callback_without_cmatvec(ccg):
    n = 128
    A, y = W.dense_system(n, 1.0, 7)
    h, h2 = ccg.Handle(), ccg.Handle()
    opd = h2.op_dense(dev(A))
    opc, _ = callback_op(ccg, h, h2, opd, n, "complex128", with_c=False)
    for method in ("cgnr", "qmr", "bicg", "cgne"):
        with pytest.raises(ccg.CcgError) as e:
            h.solve(method, opc, dev(y), dev(np.zeros(n, np.complex128)), tol=1e-10, maxit=50)
        assert e.value.status == ccg.ERR_UNSUPPORTED
    with pytest.raises(ccg.CcgError):
        h.matvec(opc, dev(y), dev(np.zeros(n, np.complex128)), trans=True)
    x = dev(np.zeros(n, np.complex128))
    st, info, _ = h.solve("bicgstab", opc, dev(y), x, tol=1e-10, maxit=200)
    assert st == 0


def test_callback_failure_ends_the_solve(ccg):
    """A callback that returns nonzero makes the solve fail with
    CCG_ERR_CUDA; the handle stays usable."""
    n = 200
    A, y = W.dense_system(n, 1.0, 8)
    h, h2 = ccg.Handle(), ccg.Handle()
    opd = h2.op_dense(dev(A))
    opc, w = callback_op(ccg, h, h2, opd, n, "complex128", fail_after=5)
    with pytest.raises(ccg.CcgError) as e:
        h.solve("bicgstab", opc, dev(y), dev(np.zeros(n, np.complex128)), tol=1e-12, maxit=500)
    assert e.value.status == ccg.ERR_CUDA
    assert "callback" in str(e.value)
    opb = h.op_dense(dev(A))
    x = dev(np.zeros(n, np.complex128))
    st, info, _ = h.solve("bicgstab", opb, dev(y), x, tol=1e-10, maxit=500)
    assert st == 0 and info["true_relres"] <= 1e-9


def test_callback_refined(ccg):
    """Refinement with callback operators on both sides (complex128 residual,
    complex64 inner solve): the same solution as with the built-in operators."""
    n = 512
    A, y = W.dense_system(n, 3.0, 0)
    h, h2 = ccg.Handle(), ccg.Handle()
    A64, A32 = dev(A), dev(A.astype(np.complex64))
    d64, d32 = h2.op_dense(A64), h2.op_dense(A32)
    c64, _ = callback_op(ccg, h, h2, d64, n, "complex128")
    c32, _ = callback_op(ccg, h, h2, d32, n, "complex64")
    b64, b32 = h.op_dense(A64), h.op_dense(A32)
    xs = []
    for op, op_in in ((c64, c32), (b64, b32)):
        x = dev(np.zeros(n, np.complex128))
        st, info, hist, inner = h.solve_refined("bicgstab", op, op_in, dev(y), x, tol=1e-10)
        assert st == 0 and info["true_relres"] <= 1e-10
        xs.append(x.cpu().numpy())
    assert relerr(xs[0], xs[1]) < 1e-13


def test_callback_dipole_cocg(ccg):
    """The dipole operator behind callbacks (complex symmetric, flagged):
    COCG iterates equal the built-in operator's."""
    occ = W.sphere_occupancy(8)
    kd, m = 0.5, 1.5 + 0.01j
    h, h2 = ccg.Handle(), ccg.Handle()
    dip2 = h2.op_dipole(occ, kd, m)
    n = dip2.n
    opc, _ = callback_op(ccg, h, h2, dip2, n, "complex128", symmetric=True)
    dip = h.op_dipole(occ, kd, m)
    y = W.plane_wave_rhs(occ, kd)
    xs = []
    for op in (opc, dip):
        x = dev(np.zeros(n, np.complex128))
        h.solve("cocg", op, dev(y), x, tol=0.0, maxit=15)
        xs.append(x.cpu().numpy())
    assert relerr(xs[0], xs[1]) < 1e-12
