"""GPU parity of the dense hot path against the CPU oracle, through the C ABI.

Rows covered: dense A x and A^H x sweeps, conjugated and unconjugated dot
products, and the fused per-method updates of BiCGSTAB, CGNR, QMR and COCG
(the manual's Sec. 2.1 and Sec. 2.2 methods on the Sec. 1 problem).

Tolerances:
  * complex128: iterates x_k after k iterations within 1e-9 relative of the
    oracle's (the two differ only in summation order); final recurrence
    residual <= 1e-10 and equal iteration counts.
  * complex64: matrix-vector products within 1e-5 relative (single-precision
    accumulation over up to n terms); solves reach relative residual 1e-6
    (true residual computed by the oracle in double).
"""
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


@pytest.fixture(scope="module")
def h(ccg):
    return ccg.Handle()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def vec_ok(got, ref, dtype):
    tol = 1e-12 if dtype == np.complex128 else 2e-5
    return np.abs(got - ref).max() <= tol * max(np.abs(ref).max(), 1e-300)


# ---------------------------------------------------------------- operators
@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
@pytest.mark.parametrize("n", [1, 2, 7, 33, 128, 255, 256, 1000, 1025, 4099])
def test_matvec_n_and_c(h, dtype, n):
    A, _ = W.dense_system(n, 1.0, n, dtype=dtype)
    x = W.random_vector(n, n + 1, dtype)
    op = h.op_dense(dev(A))
    oop = O.DenseOp(A)
    for trans in (False, True):
        yd = torch.empty(n, dtype=getattr(torch, np.dtype(dtype).name), device="cuda")
        h.matvec(op, dev(x), yd, trans=trans)
        torch.cuda.synchronize()
        assert vec_ok(yd.cpu().numpy(), oop.matvec(x, trans=trans), dtype), (n, trans)


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
def test_matvec_padded_leading_dimension(h, ccg, dtype):
    n, lda = 301, 317                       # odd lda: complex64 falls back to 8-byte loads
    A, _ = W.dense_system(lda, 1.0, 3, dtype=dtype)
    Ad = dev(A)[:n, :n]                     # row-major view with leading dimension lda
    import ctypes
    op = ctypes.c_void_p()
    code = ccg.C128 if dtype == np.complex128 else ccg.C64
    assert ccg.lib().ccg_op_dense(h.h, code, n, ctypes.c_void_p(Ad.data_ptr()), lda, 0, ctypes.byref(op)) == 0
    x = W.random_vector(n, 4, dtype)
    ref = O.DenseOp(np.ascontiguousarray(A[:n, :n]))
    for trans in (0, 1):
        yd = torch.empty(n, dtype=Ad.dtype, device="cuda")
        xd = dev(x)
        assert ccg.lib().ccg_matvec(h.h, op, trans, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr())) == 0
        torch.cuda.synchronize()
        assert vec_ok(yd.cpu().numpy(), ref.matvec(x, trans=bool(trans)), dtype)
    ccg.lib().ccg_op_destroy(op)


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
@pytest.mark.parametrize("n", [1, 5, 256, 100003])
def test_dot_products(h, dtype, n):
    u, v = W.random_vector(n, 1, dtype), W.random_vector(n, 2, dtype)
    u64, v64 = u.astype(np.complex128), v.astype(np.complex128)
    got_c = h.dot(dev(u), dev(v), conj=True)
    got_u = h.dot(dev(u), dev(v), conj=False)
    ref_c, ref_u = np.vdot(u64, v64), np.dot(u64, v64)
    scale = np.linalg.norm(u64) * np.linalg.norm(v64)
    assert abs(got_c - ref_c) <= 1e-13 * scale
    assert abs(got_u - ref_u) <= 1e-13 * scale


# ------------------------------------------------------------------ solvers
SMALL = [("bicgstab", False), ("cgnr", False), ("qmr", False), ("cocg", True), ("cocr", True), ("bicg", False),
         ("gmres", False), ("cgs", False), ("cgne", False), ("tfqmr", False), ("bicgstabl", False)]


def system(n, shift, seed, symmetric, dtype=np.complex128):
    A, y = W.dense_system(n, shift, seed)
    if symmetric:
        A = (A + A.T) / 2
    return A.astype(dtype), y.astype(dtype)


@pytest.mark.parametrize("method,sym", SMALL)
def test_iterates_match_oracle_fp64(h, method, sym):
    """x_k after k = 1..20 iterations within 1e-9 relative of the oracle's."""
    A, y = system(256, 0.6, 5, sym)        # slow enough to run 20 iterations
    x0 = W.random_vector(256, 6) * 0.1
    op = h.op_dense(dev(A), symmetric=sym)
    oop = O.DenseOp(A, symmetric=sym)
    for k in (1, 2, 3, 5, 8, 13, 20):
        ref = O.solve(oop, method, y, x0=x0, tol=0.0, maxit=k)
        xd = dev(x0.copy())
        st, info, hist = h.solve(method, op, dev(y), xd, tol=0.0, maxit=k)
        assert info["iters"] == ref.iters == k
        assert relerr(xd.cpu().numpy(), ref.x) < 1e-9, (method, k)
        assert np.allclose(hist, ref.hist, rtol=1e-9, atol=0), (method, k)


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
def test_gmres_restarts_match_oracle(h, ccg, dtype):
    """GMRES(5): iterates across several restarts, and the residual history,
    against the oracle's GMRES(5); ragged n against every tile."""
    A, y = system(1000, 1.0, 9, False, dtype)
    x0 = (W.random_vector(1000, 10) * 0.1).astype(dtype)
    h.set_option(ccg.OPT_GMRES_RESTART, 5)
    try:
        op = h.op_dense(dev(A))
        oop = O.DenseOp(A)
        tol = 1e-9 if dtype == np.complex128 else 2e-4
        for k in (1, 4, 5, 6, 11, 17):
            ref = O.solve(oop, "gmres", y, x0=x0, tol=0.0, maxit=k, restart=5)
            xd = dev(x0.copy())
            st, info, hist = h.solve("gmres", op, dev(y), xd, tol=0.0, maxit=k)
            assert info["iters"] == ref.iters == k
            assert relerr(xd.cpu().numpy(), ref.x) < tol, k
            assert np.allclose(hist, ref.hist, rtol=tol, atol=0), k
        ref = O.solve(oop, "gmres", y, tol=1e-5 if dtype == np.complex64 else 1e-10, maxit=400, restart=5)
        xd = torch.zeros(1000, dtype=xd.dtype, device="cuda")
        st, info, hist = h.solve("gmres", op, dev(y), xd, tol=1e-5 if dtype == np.complex64 else 1e-10, maxit=400)
        assert st == 0 == ref.status
        assert abs(info["iters"] - ref.iters) <= 1
    finally:
        h.set_option(ccg.OPT_GMRES_RESTART, 30)


@pytest.mark.parametrize("ell", [1, 3, 4])
def test_bicgstabl_degrees_match_oracle(h, ccg, ell):
    """BiCGstab(l) for l = 1, 3, 4 (2 is the default, in the tests above):
    iterates and residual history against the oracle's; ragged n."""
    A, y = system(1000, 0.8, 11, False)
    x0 = W.random_vector(1000, 12) * 0.1
    h.set_option(ccg.OPT_BICGSTAB_L, ell)
    try:
        op = h.op_dense(dev(A))
        oop = O.DenseOp(A)
        for k in (1, 2, 5):
            ref = O.solve(oop, "bicgstabl", y, x0=x0, tol=0.0, maxit=k, ell=ell)
            xd = dev(x0.copy())
            st, info, hist = h.solve("bicgstabl", op, dev(y), xd, tol=0.0, maxit=k)
            assert info["iters"] == ref.iters == k
            assert relerr(xd.cpu().numpy(), ref.x) < 1e-9, (ell, k)
            assert np.allclose(hist, ref.hist, rtol=1e-9, atol=0), (ell, k)
        ref = O.solve(oop, "bicgstabl", y, tol=1e-10, maxit=300, ell=ell)
        xd = torch.zeros(1000, dtype=torch.complex128, device="cuda")
        st, info, hist = h.solve("bicgstabl", op, dev(y), xd, tol=1e-10, maxit=300)
        assert st == 0 == ref.status and abs(info["iters"] - ref.iters) <= 1
        assert info["true_relres"] <= 1e-10
    finally:
        h.set_option(ccg.OPT_BICGSTAB_L, 2)


@pytest.mark.parametrize("method,sym", SMALL)
def test_small_config_solve_fp64(h, method, sym):
    """The n = 256 shift-8 system to relative residual 1e-10 (complex128)."""
    A, y = system(256, 8.0, 0, sym)
    op = h.op_dense(dev(A), symmetric=sym)
    ref = O.solve(O.DenseOp(A, symmetric=sym), method, y, tol=1e-10, maxit=1000)
    xd = torch.zeros(256, dtype=torch.complex128, device="cuda")
    st, info, hist = h.solve(method, op, dev(y), xd, tol=1e-10, maxit=1000)
    assert st == 0 and ref.status == 0
    assert info["iters"] == ref.iters
    assert info["relres"] <= 1e-10 and info["true_relres"] <= 1e-10
    assert relerr(xd.cpu().numpy(), ref.x) < 1e-9


@pytest.mark.parametrize("method,sym", SMALL)
def test_solve_fp32_reaches_1e6(h, method, sym):
    A, y = system(1000, 3.0, 2, sym, np.complex64)   # ragged against every tile
    op = h.op_dense(dev(A), symmetric=sym)
    xd = torch.zeros(1000, dtype=torch.complex64, device="cuda")
    st, info, hist = h.solve(method, op, dev(y), xd, tol=1e-6, maxit=500)
    assert st == 0
    A64, y64 = A.astype(np.complex128), y.astype(np.complex128)
    x = xd.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(y64 - A64 @ x) / np.linalg.norm(y64) < 3e-6
    ref = O.solve(O.DenseOp(A, symmetric=sym), method, y, tol=1e-6, maxit=500)
    assert abs(info["iters"] - ref.iters) <= 2


def test_full_size_matvec(h):
    """n = 8192 complex128 and complex64 products against the oracle's full
    products (the oracle finishes one in well under a second)."""
    A, _ = W.dense_system(**W.DENSE_LARGE)
    x = W.random_vector(8192, 3)
    for dtype in (np.complex128, np.complex64):
        Ah = A.astype(dtype)
        Ad = dev(Ah)
        op = h.op_dense(Ad)
        oop = O.DenseOp(Ah)
        xs = x.astype(dtype)
        for trans in (False, True):
            yd = torch.empty(8192, dtype=Ad.dtype, device="cuda")
            h.matvec(op, dev(xs), yd, trans=trans)
            torch.cuda.synchronize()
            ref = oop.matvec(xs, trans=trans)
            tol = 1e-12 if dtype == np.complex128 else 3e-5
            assert np.abs(yd.cpu().numpy() - ref).max() <= tol * np.abs(ref).max()
        del Ad, op


def test_edge_cases(h, ccg):
    n = 64
    A, y = system(n, 3.0, 1, True)
    op = h.op_dense(dev(A), symmetric=True)
    # y = 0 gives x = 0
    xd = dev(W.random_vector(n, 1))
    st, info, hist = h.solve("bicgstab", op, torch.zeros(n, dtype=torch.complex128, device="cuda"), xd, 1e-10, 50)
    assert st == 0 and info["iters"] == 0 and torch.count_nonzero(xd).item() == 0
    # maxit = 0
    xd = torch.zeros(n, dtype=torch.complex128, device="cuda")
    st, info, hist = h.solve("qmr", op, dev(y), xd, 1e-10, 0)
    assert st == ccg.NOT_CONVERGED and info["iters"] == 0
    # x0 already the solution
    xs = np.linalg.solve(A, y)
    xd = dev(xs)
    st, info, hist = h.solve("cgnr", op, dev(y), xd, 1e-10, 10)
    assert st == 0 and info["iters"] == 0
    # iteration cap
    st, info, hist = h.solve("bicgstab", op, dev(y), torch.zeros_like(xd), 1e-15, 2)
    assert st == ccg.NOT_CONVERGED and info["iters"] == 2 and len(hist) == 3
    # COCG and COCR need the symmetric flag
    op2 = h.op_dense(dev(A))
    for m in ("cocg", "cocr"):
        with pytest.raises(ccg.CcgError):
            h.solve(m, op2, dev(y), torch.zeros_like(xd), 1e-10, 10)
    # non-finite right-hand side
    yb = y.copy()
    yb[3] = np.nan
    st = None
    with pytest.raises(ccg.CcgError) as e:
        h.solve("bicgstab", op, dev(yb), torch.zeros_like(xd), 1e-10, 10)
    assert e.value.status == ccg.ERR_NONFINITE


def test_breakdowns_match_oracle(h, ccg):
    A = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    y = np.array([1, 0], dtype=np.complex128)
    op = h.op_dense(dev(A), symmetric=True)
    st, info, _ = h.solve("bicgstab", op, dev(y), torch.zeros(2, dtype=torch.complex128, device="cuda"), 1e-12, 5)
    ref = O.solve(O.DenseOp(A), "bicgstab", y, tol=1e-12, maxit=5)
    assert st == ccg.BREAKDOWN == ref.status and info["breakdown"] == ref.detail and info["iters"] == ref.iters
    I2 = np.eye(2, dtype=np.complex128)
    op = h.op_dense(dev(I2), symmetric=True)
    yb = np.array([1, 1j])
    for m in ("cocg", "cocr"):
        st, info, _ = h.solve(m, op, dev(yb), torch.zeros(2, dtype=torch.complex128, device="cuda"), 1e-12, 5)
        ref = O.solve(O.DenseOp(I2, symmetric=True), m, yb, tol=1e-12, maxit=5)
        assert st == ccg.BREAKDOWN == ref.status and info["breakdown"] == ref.detail and info["iters"] == ref.iters
    # COCR: [A r0, A r0] = 0 with [r0, A r0] != 0
    D = np.diag([1, 1j]).astype(np.complex128)
    y1 = np.array([1, 1], dtype=np.complex128)
    op = h.op_dense(dev(D), symmetric=True)
    st, info, _ = h.solve("cocr", op, dev(y1), torch.zeros(2, dtype=torch.complex128, device="cuda"), 1e-12, 5)
    ref = O.solve(O.DenseOp(D, symmetric=True), "cocr", y1, tol=1e-12, maxit=5)
    assert st == ccg.BREAKDOWN == ref.status and info["breakdown"] == ref.detail == ccg_bd_mu()
    # BiCG and CGS: <p~, A p> = 0 on the swap matrix
    op = h.op_dense(dev(A))
    for m in ("bicg", "cgs", "tfqmr", "bicgstabl"):
        st, info, _ = h.solve(m, op, dev(y), torch.zeros(2, dtype=torch.complex128, device="cuda"), 1e-12, 5)
        ref = O.solve(O.DenseOp(A), m, y, tol=1e-12, maxit=5)
        assert st == ccg.BREAKDOWN == ref.status and info["breakdown"] == ref.detail and info["iters"] == ref.iters
    # CGNE: A^H r0 = 0 with r0 != 0
    S = np.array([[1, 1], [1, 1]], dtype=np.complex128)
    y2 = np.array([1, -1], dtype=np.complex128)
    op = h.op_dense(dev(S))
    st, info, _ = h.solve("cgne", op, dev(y2), torch.zeros(2, dtype=torch.complex128, device="cuda"), 1e-12, 5)
    ref = O.solve(O.DenseOp(S), "cgne", y2, tol=1e-12, maxit=5)
    assert st == ccg.BREAKDOWN == ref.status and info["breakdown"] == ref.detail and info["iters"] == ref.iters


def ccg_bd_mu():
    return 11   # CCG_BD_MU


def test_host_buffers_equal_device_buffers(h):
    A, y = system(300, 3.0, 7, False)
    op = h.op_dense(dev(A))
    xd = torch.zeros(300, dtype=torch.complex128, device="cuda")
    h.solve("qmr", op, dev(y), xd, 1e-10, 200)
    xh = np.zeros(300, dtype=np.complex128)
    st, info, _ = h.solve("qmr", op, y.copy(), xh, 1e-10, 200)
    assert st == 0
    assert np.array_equal(xh, xd.cpu().numpy())


def test_repeat_solves_are_deterministic(h):
    A, y = system(777, 2.0, 9, False)
    op = h.op_dense(dev(A))
    outs = []
    for _ in range(2):
        xd = torch.zeros(777, dtype=torch.complex128, device="cuda")
        h.solve("bicgstab", op, dev(y), xd, 1e-10, 200)
        outs.append(xd.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
