"""The complex128 fixed-point sweep (y = A x on the integer pipe, the
default for complex128 dense operators) against exact products.

The reference sums are exact: every double is an integer times a power of
two, so each row sum is formed in Python integers at a common scale and
rounded only when compared.  The bound checked is the scheme's own,
|error| <= 2.5 n 2^(Fa + Fx - 52) per real or imaginary part, with 2^Fa the
power of two above the row's largest |re|, |im| and 2^Fx the one above the
vector's (the form of an FP64 GEMV's bound relative to the largest entries);
the tests also hold the typical error near double rounding and check the
paths that leave the integer pipe (non-finite entries) against the FP64
sweep.
"""
import math

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


def exact_parts(v):
    """Integer mantissa and exponent of every double: v = m * 2^e exactly."""
    m, e = np.frexp(v)
    return (m * 2.0 ** 53).astype(np.int64), e.astype(np.int64) - 53


def exact_matvec_error(A, x, y):
    """max over rows of |y_i - (A x)_i| / (2.5 n 2^(Fa + Fx - 52)), exactly."""
    n = A.shape[0]
    ar, ae_r = exact_parts(A.real)
    ai, ae_i = exact_parts(A.imag)
    xr, xe_r = exact_parts(x.real)
    xi, xe_i = exact_parts(x.imag)
    fx = max(math.frexp(float(v))[1] for v in np.concatenate([np.abs(x.real), np.abs(x.imag)]))
    worst = 0.0
    for i in range(n):
        base = int(min(ae_r[i].min(), ae_i[i].min()) + min(xe_r.min(), xe_i.min()))
        re = 0
        im = 0
        for j in range(n):
            p = int(ar[i, j]) * int(xr[j]) << int(ae_r[i, j] + xe_r[j] - base)
            q = int(ai[i, j]) * int(xi[j]) << int(ae_i[i, j] + xe_i[j] - base)
            re += p - q
            s = int(ar[i, j]) * int(xi[j]) << int(ae_r[i, j] + xe_i[j] - base)
            t = int(ai[i, j]) * int(xr[j]) << int(ae_i[i, j] + xe_r[j] - base)
            im += s + t
        row = np.concatenate([np.abs(A[i].real), np.abs(A[i].imag)])
        fa = max(math.frexp(float(v))[1] for v in row)
        for got, ex in ((y[i].real, re), (y[i].imag, im)):
            g_m, g_e = math.frexp(float(got))
            g_int = int(g_m * 2 ** 53)
            g_sh = g_e - 53 - base
            diff = (g_int << g_sh) - ex if g_sh >= 0 else g_int - (ex << -g_sh)
            scale = base if g_sh >= 0 else base + g_sh
            if diff == 0:
                continue
            if not any(row) or not any(x):
                return math.inf    # an exact zero product must come out exactly zero
            # log2 of |diff| 2^scale / (2.5 n 2^(fa + fx - 52)), without overflow
            lr = math.log2(abs(diff)) + scale - (math.log2(2.5 * n) + fa + fx - 52)
            worst = max(worst, 2.0 ** min(lr, 64))
    return worst


def exact_matvec_h_error(A, x, y):
    """max over columns of |y_c - (A^H x)_c| / (2.5 n 2^(Fm + Fx' - 52)),
    exactly: the A^H sweep's bound, with 2^Fm above every entry of A and
    2^Fx' above every part of x_r 2^(F_r - Fm) (F_r: row r's scale)."""
    n = A.shape[0]
    ar, ae_r = exact_parts(A.real)
    ai, ae_i = exact_parts(A.imag)
    xr, xe_r = exact_parts(x.real)
    xi, xe_i = exact_parts(x.imag)
    frow = [max(math.frexp(float(v))[1] for v in np.concatenate([np.abs(A[r].real), np.abs(A[r].imag)]))
            for r in range(n)]
    fm = max(frow)
    fx = max(math.frexp(math.ldexp(float(v), frow[r] - fm))[1]
             for r in range(n) for v in (abs(x[r].real), abs(x[r].imag)))
    base = int(min(ae_r.min(), ae_i.min()) + min(xe_r.min(), xe_i.min()))
    worst = 0.0
    for c in range(n):
        re = 0
        im = 0
        for r in range(n):
            p = int(ar[r, c]) * int(xr[r]) << int(ae_r[r, c] + xe_r[r] - base)
            q = int(ai[r, c]) * int(xi[r]) << int(ae_i[r, c] + xe_i[r] - base)
            re += p + q
            s = int(ar[r, c]) * int(xi[r]) << int(ae_r[r, c] + xe_i[r] - base)
            t = int(ai[r, c]) * int(xr[r]) << int(ae_i[r, c] + xe_r[r] - base)
            im += s - t
        for got, ex in ((y[c].real, re), (y[c].imag, im)):
            g_m, g_e = math.frexp(float(got))
            g_int = int(g_m * 2 ** 53)
            g_sh = g_e - 53 - base
            diff = (g_int << g_sh) - ex if g_sh >= 0 else g_int - (ex << -g_sh)
            scale = base if g_sh >= 0 else base + g_sh
            if diff == 0:
                continue
            lr = math.log2(abs(diff)) + scale - (math.log2(2.5 * n) + fm + fx - 52)
            worst = max(worst, 2.0 ** min(lr, 64))
    return worst


def matvec(ccg, A, x, fx, trans=False):
    h = ccg.Handle()
    h.set_option(ccg.OPT_FP64_SWEEP, fx)
    Ad = torch.from_numpy(A).cuda()
    op = h.op_dense(Ad)
    y = torch.empty(A.shape[0], dtype=torch.complex128, device="cuda")
    h.matvec(op, torch.from_numpy(x).cuda(), y, trans=trans)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("n", [1, 7, 33, 128, 257])
def test_fixed_point_within_bound(ccg, n):
    A, _ = W.dense_system(n, 3.0, n)
    x = W.random_vector(n, n + 1)
    y = matvec(ccg, A, x, 1)
    assert exact_matvec_error(A, x, y) <= 1.0
    # and near double rounding in practice: against the oracle's double sum
    ref = O.DenseOp(A).matvec(x)
    scale = np.abs(A) @ np.abs(x)
    assert np.max(np.abs(y - ref) / scale) < 1e-14


def test_fixed_point_wide_range(ccg):
    """Rows and columns scaled over 2^-300 .. 2^300, subnormal entries, a zero
    row and zero entries of x: still within the bound."""
    n = 96
    rng = np.random.default_rng(5)
    A, _ = W.dense_system(n, 1.0, 3)
    A = A * np.exp2(rng.integers(-300, 300, n))[:, None]
    A[5] = 0
    A[7, ::3] = 5e-320 + 3e-320j            # subnormal
    A[9] *= np.exp2(rng.integers(-40, 40, n))
    x = W.random_vector(n, 4)
    x[::7] = 0
    x[3] *= 2.0 ** 60
    y = matvec(ccg, A, x, 1)
    assert np.all(y[5] == 0)
    assert exact_matvec_error(A, x, y) <= 1.0


@pytest.mark.parametrize("n", [1, 7, 129, 300])
def test_fixed_point_adjoint_within_bound(ccg, n):
    """A^H x on the integer pipe (the row-scaled vector's digits against the
    operator's): within its bound, and near double rounding in practice."""
    A, _ = W.dense_system(n, 3.0, n + 40)
    x = W.random_vector(n, n + 41)
    y = matvec(ccg, A, x, 1, trans=True)
    assert exact_matvec_h_error(A, x, y) <= 1.0
    ref = O.DenseOp(A).matvec(x, trans=True)
    scale = np.abs(A).T @ np.abs(x)
    assert np.max(np.abs(y - ref) / scale) < 1e-14


def test_fixed_point_adjoint_wide_range(ccg):
    """Rows over 2^-300 .. 2^300 (the row scales folded into the vector),
    subnormal entries, a zero row, zero entries of x: within the bound."""
    n = 80
    rng = np.random.default_rng(15)
    A, _ = W.dense_system(n, 1.0, 4)
    A = A * np.exp2(rng.integers(-300, 300, n))[:, None]
    A[5] = 0
    A[7, ::3] = 5e-320 + 3e-320j
    x = W.random_vector(n, 5)
    x[::7] = 0
    x[3] *= 2.0 ** 60
    y = matvec(ccg, A, x, 1, trans=True)
    assert exact_matvec_h_error(A, x, y) <= 1.0


def test_non_finite_takes_the_fp64_pipe(ccg):
    n = 200
    A, _ = W.dense_system(n, 3.0, 8)
    x = W.random_vector(n, 9)
    # a non-finite vector entry: the sweep sums those rows on the FP64 pipe
    xb = x.copy()
    xb[17] = np.inf
    y1, y0 = matvec(ccg, A, xb, 1), matvec(ccg, A, xb, 0)
    assert np.array_equal(np.isnan(y1), np.isnan(y0)) and np.array_equal(np.isinf(y1), np.isinf(y0))
    fin = np.isfinite(y0)
    assert np.allclose(y1[fin], y0[fin], rtol=1e-13, atol=0)
    # a non-finite matrix entry: flagged when the digits are made, every
    # sweep of that operator takes the FP64 pipe
    Ab = A.copy()
    Ab[3, 4] = np.nan
    y1, y0 = matvec(ccg, Ab, x, 1), matvec(ccg, Ab, x, 0)
    assert np.array_equal(np.isnan(y1), np.isnan(y0)) and np.isnan(y1[3]) and np.isfinite(y1[4])
    fin = np.isfinite(y0)
    assert np.allclose(y1[fin], y0[fin], rtol=1e-13, atol=0)
    # the same for A^H x (the column-tiled sweep): an infinite x_17 reaches
    # every column; a NaN at A[3, 4] only column 4
    for Ax, xx, some_finite in ((A, xb, False), (Ab, x, True)):
        y1, y0 = matvec(ccg, Ax, xx, 1, trans=True), matvec(ccg, Ax, xx, 0, trans=True)
        assert np.array_equal(np.isnan(y1), np.isnan(y0)) and np.array_equal(np.isinf(y1), np.isinf(y0))
        fin = np.isfinite(y0)
        assert fin.any() == some_finite and np.allclose(y1[fin], y0[fin], rtol=1e-13, atol=0)
    assert np.isnan(y1[4]) and np.isfinite(y1[3])


def test_fixed_point_solves_match_oracle(ccg):
    """complex128 solves on the fixed-point sweeps (A x and A^H x; QMR and
    BiCG take their A p and A^H q from the two): whole solves against the
    oracle (x to 1e-9) with the integer and the FP64 sweeps."""
    n = 1000
    A, y = W.dense_system(n, 3.0, 21)
    for m in ("bicgstab", "cgnr", "qmr", "bicg", "cgne"):
        ref = O.solve(O.DenseOp(A), m, y, tol=1e-10, maxit=300)
        for fx in (1, 0):
            h = ccg.Handle()
            h.set_option(ccg.OPT_FP64_SWEEP, fx)
            op = h.op_dense(torch.from_numpy(A).cuda())
            xd = torch.zeros(n, dtype=torch.complex128, device="cuda")
            st, info, hist = h.solve(m, op, torch.from_numpy(y).cuda(), xd, tol=1e-10, maxit=300)
            assert st == 0 and info["iters"] == ref.iters and info["true_relres"] <= 1e-10
            assert np.linalg.norm(xd.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x), (m, fx)


@pytest.mark.parametrize("n", [33, 1000])
def test_fixed_point_padded_rows(ccg, n):
    """An operator whose rows are padded (lda = n + 5): the digits are made
    from the strided rows, so A x and A^H x are bitwise those of the
    contiguous matrix, and a CGNR solve (both sweeps) matches the oracle."""
    A, y = W.dense_system(n, 3.0, n + 7)
    x = W.random_vector(n, n + 8)
    store = np.zeros((n, n + 5), dtype=np.complex128)
    store[:, :n] = A
    h = ccg.Handle()
    Ad = torch.from_numpy(A).cuda()
    Sd = torch.from_numpy(store).cuda()
    op_c = h.op_dense(Ad)
    op_p = h.op_dense(Sd[:, :n])
    xd = torch.from_numpy(x).cuda()
    for trans in (False, True):
        yc = torch.empty(n, dtype=torch.complex128, device="cuda")
        yp = torch.empty_like(yc)
        h.matvec(op_c, xd, yc, trans=trans)
        h.matvec(op_p, xd, yp, trans=trans)
        torch.cuda.synchronize()
        assert torch.equal(yc, yp), trans
    ref = O.solve(O.DenseOp(A), "cgnr", y, tol=1e-10, maxit=300)
    xs = torch.zeros(n, dtype=torch.complex128, device="cuda")
    st, info, _ = h.solve("cgnr", op_p, torch.from_numpy(y).cuda(), xs, tol=1e-10, maxit=300)
    assert st == 0 and info["iters"] == ref.iters
    assert np.linalg.norm(xs.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
