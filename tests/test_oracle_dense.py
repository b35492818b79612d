"""Pins of the CPU oracle's dense-operator solvers against what mathematics and
independent libraries fix (no GPU).

The manual (Sec. 2.1, Sec. 2.2) names the methods but prints no recurrences,
iterates or worked examples, so every pin here is a property of the method
or an independent implementation of the same textbook algorithm:
  * LAPACK (numpy.linalg.solve) on small systems;
  * scipy's BiCGSTAB / QMR / CG / BiCG / MINRES iterates (independent code,
    same conventions: shadow vector r_0, conjugated products);
  * each Krylov method's defining condition solved directly on tiny systems
    (x_k - x_0 in K_k(A, r_0) and the residual orthogonal to the method's
    test space), iterate by iterate;
  * finite termination, eigenvalue-count termination on diagonal operators,
    CGNR's monotone residual, QMR's quasi-residual bound, breakdown cases.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import oracle as O
from paper_1208_4869_gb300 import workloads as W

METHODS = ["bicgstab", "cgnr", "qmr"]
SYM = ("cocg", "cocr")                 # methods for complex-symmetric A
ALL = METHODS + ["cocg", "cocr", "bicg", "gmres", "cgs", "cgne", "tfqmr", "bicgstabl"]


def relres(A, x, y):
    return np.linalg.norm(y - A @ x) / np.linalg.norm(y)


@pytest.mark.parametrize("dtype,tol", [(np.complex128, 1e-13), (np.complex64, 2e-6)])
def test_dense_matvec_matches_numpy(dtype, tol):
    A, _ = W.dense_system(37, 1.0, 3, dtype=dtype)
    x = W.random_vector(37, 4, dtype)
    op = O.DenseOp(A)
    ref = A.astype(np.complex128) @ x.astype(np.complex128)
    refh = A.astype(np.complex128).conj().T @ x.astype(np.complex128)
    assert np.abs(op.matvec(x) - ref).max() / np.abs(ref).max() < tol
    assert np.abs(op.matvec(x, trans=True) - refh).max() / np.abs(refh).max() < tol


@pytest.mark.parametrize("method", ALL)
def test_solution_matches_lapack(method):
    n = 48
    A, y = W.dense_system(n, 2.0, 11)
    if method in SYM:
        A = (A + A.T) / 2
    xs = np.linalg.solve(A, y)
    op = O.DenseOp(A, symmetric=(method in SYM))
    r = O.solve(op, method, y, tol=1e-12, maxit=500)
    assert r.status == O.OK
    assert np.linalg.norm(r.x - xs) / np.linalg.norm(xs) < 1e-10
    assert r.hist[-1] <= 1e-12
    assert abs(relres(A, r.x, y) - r.hist[-1]) < 1e-12


@pytest.mark.parametrize("method,fn", [("bicgstab", sla.bicgstab), ("qmr", sla.qmr)])
def test_iterates_match_scipy(method, fn):
    """scipy's BiCGSTAB and QMR (Templates forms) are independent code with the
    same shadow vector r^ = r_0 and conjugated products."""
    A, y = W.dense_system(64, 1.0, 7)
    x0 = W.random_vector(64, 8)
    xs = []
    fn(A, y, x0=x0.copy(), rtol=1e-15, atol=0.0, maxiter=10, callback=lambda xk: xs.append(xk.copy()))
    op = O.DenseOp(A)
    for k in range(1, 9):
        r = O.solve(op, method, y, x0=x0, tol=0.0, maxit=k)
        assert r.iters == k
        assert np.linalg.norm(r.x - xs[k - 1]) / np.linalg.norm(xs[k - 1]) < 1e-12


def test_cgnr_iterates_match_cg_on_normal_equations():
    """CGNR is CG on A^H A x = A^H y; scipy's CG on that Hermitian matrix gives
    the same iterates in exact arithmetic."""
    A, y = W.dense_system(40, 1.0, 5)
    N = A.conj().T @ A
    b = A.conj().T @ y
    xs = []
    sla.cg(N, b, rtol=1e-15, atol=0.0, maxiter=8, callback=lambda xk: xs.append(xk.copy()))
    op = O.DenseOp(A)
    for k in range(1, 7):
        r = O.solve(op, "cgnr", y, tol=0.0, maxit=k)
        assert np.linalg.norm(r.x - xs[k - 1]) / np.linalg.norm(xs[k - 1]) < 1e-11


def test_cocg_is_cg_on_real_spd():
    """With real SPD A and real y the unconjugated form equals textbook CG."""
    rng = np.random.default_rng(1)
    B = rng.standard_normal((40, 40))
    S = B @ B.T + 40 * np.eye(40)
    b = rng.standard_normal(40)
    xs = []
    sla.cg(S, b, rtol=1e-15, atol=0.0, maxiter=8, callback=lambda xk: xs.append(xk.copy()))
    op = O.DenseOp(S.astype(np.complex128), symmetric=True)
    for k in range(1, 7):
        r = O.solve(op, "cocg", b.astype(np.complex128), tol=0.0, maxit=k)
        assert np.linalg.norm(r.x - xs[k - 1]) / np.linalg.norm(xs[k - 1]) < 1e-12
        assert np.abs(r.x.imag).max() == 0.0


def test_cocg_differs_from_conjugated_cg_on_complex_symmetric():
    """On a complex-symmetric non-Hermitian A, COCG must converge (its theory
    holds) and its first iterate uses the unconjugated [r, r] / [p, Ap]."""
    A, y = W.dense_system(30, 3.0, 9)
    A = (A + A.T) / 2
    op = O.DenseOp(A, symmetric=True)
    r1 = O.solve(op, "cocg", y, tol=0.0, maxit=1)
    alpha = (y @ y) / (y @ (A @ y))          # first step from x0 = 0: p = r = y
    assert np.allclose(r1.x, alpha * y, rtol=1e-13, atol=0)
    r = O.solve(op, "cocg", y, tol=1e-11, maxit=200)
    assert r.status == O.OK and relres(A, r.x, y) < 1e-10


@pytest.mark.parametrize("method", ALL)
def test_finite_termination_small(method):
    """Exact arithmetic ends in at most n steps; in floating point the relative
    residual after n steps (n+1 for CGNR) is tiny on a well-conditioned system."""
    n = 6
    A, y = W.dense_system(n, 4.0, 21)
    if method in SYM:
        A = (A + A.T) / 2
    op = O.DenseOp(A, symmetric=(method in SYM))
    steps = n + 1 if method in ("cgnr", "cgne") else n
    r = O.solve(op, method, y, tol=0.0, maxit=steps)
    assert relres(A, r.x, y) < 1e-8


@pytest.mark.parametrize("method", ALL)
def test_diagonal_operator_distinct_eigenvalues(method):
    """A diagonal A with d distinct eigenvalues (distinct moduli, so A^H A has d
    distinct eigenvalues too) and a RHS with every component nonzero: the
    Krylov space has dimension d, so the method converges at step d."""
    lam = np.array([1.0 + 0.5j, 2.0 - 1.0j, 3.5 + 0.2j, 5.0 + 3.0j])
    diag = np.repeat(lam, 5)
    A = np.diag(diag).astype(np.complex128)
    y = W.random_vector(len(diag), 3)
    op = O.DenseOp(A, symmetric=True)
    r = O.solve(op, method, y, tol=1e-10, maxit=50)
    assert r.status == O.OK
    # BiCGstab(2): an iteration is two BiCG steps
    assert r.iters == (len(lam) + 1) // 2 if method == "bicgstabl" else r.iters == len(lam)
    assert relres(A, r.x, y) < 1e-10


def test_cgnr_terminates_in_distinct_moduli():
    """CGNR works on A^H A: eigenvalues of equal modulus collapse."""
    lam = np.array([1.0, 1.0j, 2.0, -2.0j + 0.0, 3.0])   # moduli 1, 1, 2, 2, 3 -> 3 distinct
    A = np.diag(np.repeat(lam, 4)).astype(np.complex128)
    y = W.random_vector(A.shape[0], 4)
    r = O.solve(O.DenseOp(A), "cgnr", y, tol=1e-10, maxit=50)
    assert r.status == O.OK and r.iters == 3
    r_b = O.solve(O.DenseOp(A), "bicgstab", y, tol=1e-10, maxit=50)
    assert r_b.iters == 5


def test_cgnr_residual_monotone():
    """CGNR minimises ||y - A x|| over its Krylov space, so the residual never grows."""
    A, y = W.dense_system(96, 0.3, 4)
    r = O.solve(O.DenseOp(A), "cgnr", y, tol=1e-12, maxit=400)
    h = r.hist
    assert len(h) > 20
    assert np.all(np.diff(h) <= 1e-14 * h[:-1])


def test_qmr_quasi_residual_bound():
    """||r_i|| <= sqrt(i+1) tau_i, the quasi-minimal residual bound."""
    A, y = W.dense_system(96, 0.3, 4)
    r = O.solve(O.DenseOp(A), "qmr", y, tol=1e-12, maxit=400, want_tau=True)
    yn = np.linalg.norm(y)
    i = np.arange(len(r.hist))
    assert len(r.hist) > 20
    assert np.all(r.hist * yn <= np.sqrt(i + 1) * r.tau * (1 + 1e-10))


@pytest.mark.parametrize("method", ALL)
def test_identity_converges_in_one(method):
    n = 20
    A = np.eye(n, dtype=np.complex128)
    y = W.random_vector(n, 2)
    r = O.solve(O.DenseOp(A, symmetric=True), method, y, tol=1e-12, maxit=10)
    assert r.status == O.OK and r.iters == 1
    assert np.allclose(r.x, y, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("method", ALL)
def test_zero_rhs(method):
    A, _ = W.dense_system(10, 1.0, 1)
    A = (A + A.T) / 2
    x0 = W.random_vector(10, 5)
    r = O.solve(O.DenseOp(A, symmetric=True), method, np.zeros(10, complex), x0=x0, tol=1e-10, maxit=10)
    assert r.status == O.OK and r.iters == 0
    assert np.all(r.x == 0)


def test_breakdowns():
    # BiCGSTAB: sigma = <r^, A p> = 0 on the swap matrix with y = e_1.
    A = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    r = O.solve(O.DenseOp(A), "bicgstab", np.array([1, 0], dtype=complex), tol=1e-12, maxit=5)
    assert r.status == O.BREAKDOWN and r.detail == 2 and r.iters == 0
    # COCG: [r0, r0] = 1 + i^2 = 0 with r0 != 0.
    r = O.solve(O.DenseOp(np.eye(2, dtype=complex), symmetric=True), "cocg", np.array([1, 1j]), tol=1e-12, maxit=5)
    assert r.status == O.BREAKDOWN and r.detail == 1
    # COCG and COCR refuse an operator not marked symmetric.
    A, y = W.dense_system(8, 1.0, 1)
    for m in SYM:
        r = O.solve(O.DenseOp(A), m, y, tol=1e-12, maxit=5)
        assert r.status == O.INVALID
    # COCR: [r0, A r0] = 0 with A = I and r0 = (1, i).
    r = O.solve(O.DenseOp(np.eye(2, dtype=complex), symmetric=True), "cocr", np.array([1, 1j]), tol=1e-12, maxit=5)
    assert r.status == O.BREAKDOWN and r.detail == 1 and r.iters == 0
    # COCR: [q, q] = [A r0, A r0] = 0 while [r0, A r0] != 0 (A = diag(1, i), r0 = (1, 1)):
    # A r0 = (1, i), [r0, A r0] = 1 + i, [A r0, A r0] = 1 - 1 = 0.
    r = O.solve(O.DenseOp(np.diag([1, 1j]).astype(complex), symmetric=True), "cocr", np.array([1, 1], complex),
                tol=1e-12, maxit=5)
    assert r.status == O.BREAKDOWN and r.detail == 11 and r.iters == 0
    # GMRES: a zero Hessenberg column (A = 0) leaves the projected system singular.
    r = O.solve(O.DenseOp(np.zeros((4, 4), complex)), "gmres", np.ones(4, complex), tol=1e-12, maxit=5)
    assert r.status == O.BREAKDOWN and r.detail == 12 and r.iters == 0
    # BiCG and CGS: sigma = <p~, A p> = 0 on the swap matrix with y = e_1.
    A = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    for m in ("bicg", "cgs", "tfqmr", "bicgstabl"):
        r = O.solve(O.DenseOp(A), m, np.array([1, 0], dtype=complex), tol=1e-12, maxit=5)
        assert r.status == O.BREAKDOWN and r.detail == 2 and r.iters == 0
    # CGNE: p = A^H r0 = 0 with r0 != 0 (r0 in the null space of A^H).
    A = np.array([[1, 1], [1, 1]], dtype=np.complex128)
    r = O.solve(O.DenseOp(A), "cgne", np.array([1, -1], dtype=complex), tol=1e-12, maxit=5)
    assert r.status == O.BREAKDOWN and r.detail == 6 and r.iters == 0


def test_maxit_not_converged():
    A, y = W.dense_system(64, 0.2, 2)
    r = O.solve(O.DenseOp(A), "bicgstab", y, tol=1e-14, maxit=3)
    assert r.status == O.NOT_CONVERGED and r.iters == 3 and len(r.hist) == 4


def test_bicgstab_half_step_exit():
    """When ||s|| meets the tolerance the update x += alpha p ends the solve,
    counted as one iteration; A = 2 I reaches it at the first half step."""
    A = 2 * np.eye(8, dtype=np.complex128)
    y = W.random_vector(8, 1)
    r = O.solve(O.DenseOp(A), "bicgstab", y, tol=1e-12, maxit=5)
    assert r.iters == 1 and r.status == O.OK
    assert np.allclose(r.x, y / 2, rtol=1e-15, atol=0)


@pytest.mark.parametrize("method", METHODS)
def test_single_precision_reaches_1e6(method):
    A, y = W.dense_system(256, 8.0, 0, dtype=np.complex64)
    r = O.solve(O.DenseOp(A), method, y, tol=1e-6, maxit=200)
    assert r.status == O.OK
    A64 = A.astype(np.complex128)
    assert relres(A64, r.x.astype(np.complex128), y.astype(np.complex128)) < 3e-6


def test_small_config_iteration_counts():
    """The n=256 shift-8 system converges fast; record the counts the GPU must match."""
    A, y = W.dense_system(**W.DENSE_SMALL)
    op = O.DenseOp(A)
    its = {m: O.solve(op, m, y, tol=1e-10, maxit=1000).iters for m in METHODS}
    assert all(3 <= v <= 30 for v in its.values()), its


# ---- the methods' defining conditions, solved directly -----------------------
def krylov_basis(A, v, k):
    """Orthonormal basis of K_k(A, v) = span{v, A v, ..., A^(k-1) v}."""
    V = np.empty((len(v), k), dtype=np.complex128)
    w = v.copy()
    for j in range(k):
        V[:, j] = w
        w = A @ w
    return np.linalg.qr(V)[0]


def galerkin_iterate(method, A, y, x0, k):
    """x_k = x_0 + V c, V spanning K_k(A, r_0), with the residual r_k = r_0 - A V c
    orthogonal to the method's test space:
      COCG  [v, r_k] = 0 for v in K_k(A, r_0)          (v^T r_k, A = A^T)
      COCR  [A v, r_k] = 0 for v in K_k(A, r_0)        ((A v)^T r_k)
      BiCG  <w, r_k> = 0 for w in K_k(A^H, r_0)        (w^H r_k)"""
    r0 = y - A @ x0
    V = krylov_basis(A, r0, k)
    if method == "cocg":
        T = V.T
    elif method == "cocr":
        T = (A @ V).T
    else:
        T = krylov_basis(A.conj().T, r0, k).conj().T
    c = np.linalg.solve(T @ (A @ V), T @ r0)
    return x0 + V @ c


@pytest.mark.parametrize("method", ["cocg", "cocr", "bicg"])
def test_iterates_satisfy_the_defining_condition(method):
    n = 40
    A, y = W.dense_system(n, 3.0, 13)
    if method in SYM:
        A = (A + A.T) / 2
    x0 = W.random_vector(n, 14)
    op = O.DenseOp(A, symmetric=(method in SYM))
    for k in range(1, 7):
        r = O.solve(op, method, y, x0=x0, tol=0.0, maxit=k)
        assert r.iters == k
        xk = galerkin_iterate(method, A, y, x0, k)
        assert np.linalg.norm(r.x - xk) / np.linalg.norm(xk) < 1e-10, (method, k)


def test_galerkin_pin_catches_a_conjugated_form():
    """The COCR condition is not met by the conjugated variant (conjugate
    residual with <., .>): a dropped-conjugate mistake would fail the pin."""
    n = 40
    A, y = W.dense_system(n, 3.0, 13)
    A = (A + A.T) / 2
    x0 = np.zeros(n, complex)
    r0 = y - A @ x0
    V = krylov_basis(A, r0, 3)
    AV = A @ V
    c = np.linalg.solve(AV.conj().T @ AV, AV.conj().T @ r0)      # minimal residual (conjugated)
    wrong = x0 + V @ c
    assert np.linalg.norm(wrong - galerkin_iterate("cocr", A, y, x0, 3)) > 1e-6 * np.linalg.norm(wrong)


def test_cocr_is_minres_on_real_spd():
    """With real SPD A and real y, COCR is the conjugate residual method, whose
    iterates equal MINRES's (scipy, independent code); its residual decreases."""
    rng = np.random.default_rng(2)
    B = rng.standard_normal((40, 40))
    S = B @ B.T + 40 * np.eye(40)
    b = rng.standard_normal(40)
    xs = []
    sla.minres(S, b, rtol=1e-15, maxiter=8, callback=lambda xk: xs.append(xk.copy()))
    op = O.DenseOp(S.astype(np.complex128), symmetric=True)
    for k in range(1, 7):
        r = O.solve(op, "cocr", b.astype(np.complex128), tol=0.0, maxit=k)
        assert np.linalg.norm(r.x - xs[k - 1]) / np.linalg.norm(xs[k - 1]) < 1e-11
        assert np.abs(r.x.imag).max() == 0.0
    r = O.solve(op, "cocr", b.astype(np.complex128), tol=1e-12, maxit=100)
    assert np.all(np.diff(r.hist) <= 0)


def test_bicg_iterates_match_scipy():
    """scipy's BiCG (independent code): shadow r~_0 = r_0, A^H, conjugated products."""
    A, y = W.dense_system(64, 1.0, 7)
    x0 = W.random_vector(64, 8)
    xs = []
    sla.bicg(A, y, x0=x0.copy(), rtol=1e-15, atol=0.0, maxiter=10, callback=lambda xk: xs.append(xk.copy()))
    op = O.DenseOp(A)
    for k in range(1, 9):
        r = O.solve(op, "bicg", y, x0=x0, tol=0.0, maxit=k)
        assert r.iters == k
        assert np.linalg.norm(r.x - xs[k - 1]) / np.linalg.norm(xs[k - 1]) < 1e-12


def minres_iterate(A, y, x0, k):
    """argmin ||y - A x|| over x in x0 + K_k(A, r_0), by least squares."""
    r0 = y - A @ x0
    V = krylov_basis(A, r0, k)
    c = np.linalg.lstsq(A @ V, r0, rcond=None)[0]
    return x0 + V @ c


def test_gmres_first_cycle_is_the_least_squares_minimiser():
    """Iterate k of a cycle minimises the residual over x0 + K_k(A, r0); its
    recorded residual is that minimum (the Givens estimate is exact)."""
    n = 40
    A, y = W.dense_system(n, 2.0, 15)
    x0 = W.random_vector(n, 16)
    op = O.DenseOp(A)
    for k in range(1, 8):
        r = O.solve(op, "gmres", y, x0=x0, tol=0.0, maxit=k, restart=30)
        assert r.iters == k
        xk = minres_iterate(A, y, x0, k)
        assert np.linalg.norm(r.x - xk) / np.linalg.norm(xk) < 1e-10, k
        assert abs(r.hist[k] - relres(A, xk, y)) < 1e-12
    # the ordering of the residuals is that of a minimiser over growing spaces
    r = O.solve(op, "gmres", y, x0=x0, tol=0.0, maxit=12, restart=30)
    assert np.all(np.diff(r.hist) <= 1e-15)


def test_gmres_restarts_from_the_cycle_end():
    """GMRES(3): after a cycle, x_3 is the minimiser over x0 + K_3; the next
    cycle minimises over x_3 + K_j(A, y - A x_3)."""
    n = 40
    A, y = W.dense_system(n, 2.0, 17)
    x0 = W.random_vector(n, 18)
    op = O.DenseOp(A)
    x3 = minres_iterate(A, y, x0, 3)
    for k, want in [(3, x3), (4, minres_iterate(A, y, x3, 1)), (5, minres_iterate(A, y, x3, 2)),
                    (6, minres_iterate(A, y, x3, 3))]:
        r = O.solve(op, "gmres", y, x0=x0, tol=0.0, maxit=k, restart=3)
        assert r.iters == k and r.status == O.NOT_CONVERGED
        assert np.linalg.norm(r.x - want) / np.linalg.norm(want) < 1e-10, k
    r = O.solve(op, "gmres", y, x0=x0, tol=1e-12, maxit=400, restart=3)
    assert r.status == O.OK and np.all(np.diff(r.hist) <= 1e-15)
    assert relres(A, r.x, y) < 1e-11


def test_cgs_iterates_match_scipy():
    """scipy's CGS (independent code): shadow r^ = r_0, conjugated products."""
    A, y = W.dense_system(64, 1.5, 19)
    x0 = W.random_vector(64, 20)
    xs = []
    sla.cgs(A, y, x0=x0.copy(), rtol=1e-15, atol=0.0, maxiter=10, callback=lambda xk: xs.append(xk.copy()))
    op = O.DenseOp(A)
    for k in range(1, 9):
        r = O.solve(op, "cgs", y, x0=x0, tol=0.0, maxit=k)
        assert r.iters == k
        assert np.linalg.norm(r.x - xs[k - 1]) / np.linalg.norm(xs[k - 1]) < 1e-11


def test_cgne_is_cg_on_the_adjoint_normal_equations():
    """CGNE is CG on A A^H u = r_0 with x = x_0 + A^H u (scipy's CG on that
    Hermitian matrix, independent code); its error ||x* - x_k|| decreases."""
    A, y = W.dense_system(40, 1.0, 23)
    x0 = W.random_vector(40, 24)
    r0 = y - A @ x0
    us = []
    sla.cg(A @ A.conj().T, r0, rtol=1e-15, atol=0.0, maxiter=8, callback=lambda uk: us.append(uk.copy()))
    op = O.DenseOp(A)
    xstar = np.linalg.solve(A, y)
    errs = []
    for k in range(1, 7):
        r = O.solve(op, "cgne", y, x0=x0, tol=0.0, maxit=k)
        want = x0 + A.conj().T @ us[k - 1]
        assert np.linalg.norm(r.x - want) / np.linalg.norm(want) < 1e-11
        errs.append(np.linalg.norm(r.x - xstar))
    assert np.all(np.diff(errs) < 0)


def test_tfqmr_iterates_match_scipy():
    """scipy's TFQMR (independent code) calls back after every half-step; an
    iteration here is two half-steps (two products)."""
    A, y = W.dense_system(64, 1.5, 19)
    x0 = W.random_vector(64, 20)
    xs = []
    sla.tfqmr(A, y, x0=x0.copy(), rtol=1e-15, atol=0.0, maxiter=20, callback=lambda xk: xs.append(xk.copy()))
    op = O.DenseOp(A)
    for k in range(1, 8):
        r = O.solve(op, "tfqmr", y, x0=x0, tol=0.0, maxit=k)
        assert r.iters == k
        assert np.linalg.norm(r.x - xs[2 * k - 1]) / np.linalg.norm(xs[2 * k - 1]) < 1e-12
        # the recorded quantity bounds the true residual
        assert relres(A, r.x, y) <= r.hist[k] * (1 + 1e-12)


def test_bicgstab1_is_bicgstab():
    """BiCGstab(1) is BiCGSTAB: scipy's BiCGSTAB iterates (independent code)."""
    A, y = W.dense_system(64, 1.0, 7)
    x0 = W.random_vector(64, 8)
    xs = []
    sla.bicgstab(A, y, x0=x0.copy(), rtol=1e-15, atol=0.0, maxiter=10, callback=lambda xk: xs.append(xk.copy()))
    op = O.DenseOp(A)
    for k in range(1, 7):
        r = O.solve(op, "bicgstabl", y, x0=x0, tol=0.0, maxit=k, ell=1)
        assert np.linalg.norm(r.x - xs[k - 1]) / np.linalg.norm(xs[k - 1]) < 1e-12


@pytest.mark.parametrize("ell", [2, 3, 4])
def test_bicgstabl_first_cycle_from_its_definition(ell):
    """After one cycle from x0, BiCGstab(l) is the BiCG iterate of step l,
    s = y - A x_l (Petrov-Galerkin, solved directly), corrected by the
    degree-l minimal-residual polynomial: r = s - sum_j g_j A^j s with g
    minimising ||r|| (least squares), x = x_l + sum_j g_j A^(j-1) s."""
    n = 40
    A, y = W.dense_system(n, 2.0, 25)
    x0 = W.random_vector(n, 26)
    xb = galerkin_iterate("bicg", A, y, x0, ell)
    s = y - A @ xb
    K = [s]
    for _ in range(ell):
        K.append(A @ K[-1])
    g = np.linalg.lstsq(np.stack(K[1:], axis=1), s, rcond=None)[0]
    want = xb + sum(g[j] * K[j] for j in range(ell))
    r = O.solve(O.DenseOp(A), "bicgstabl", y, x0=x0, tol=0.0, maxit=1, ell=ell)
    assert r.iters == 1
    assert np.linalg.norm(r.x - want) / np.linalg.norm(want) < 1e-10
    assert abs(r.hist[1] - relres(A, want, y)) < 1e-11
