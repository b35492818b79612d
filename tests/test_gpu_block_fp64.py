"""FP64-accurate complex128 block products on the tensor cores (integer digit
slices, exact bf16 products, fp32 level sums, int64 combination) through
the C ABI, against exact rational references.

The product Y = A X is the manual's `matvec` (Sec. 5) applied to a block of
right-hand sides.  Bounds, with K = 2n real terms per entry:
  * rigorous: |y - exact| <= K 2^-52 max|a_i.| max|x_.c| + 2^-52 |exact|
    (8 seven-bit digits per operand keep 56 bits; the dropped digit pairs
    and remainders are below 2^-54.5 of 2^(e_i + f_c) per term, and
    2^(e_i + f_c) < 4 max|a_i.| max|x_.c|), the bound an FP64 GEMM obeys;
  * typical, for random signs: |y - exact| <= sqrt(K) 2^-50 max|a| max|x|
    + 2^-52 |exact|, far below what a lost digit level would leave;
  * the adversarial block whose digits all sit at their bounds with equal
    signs drives level sums of a K = 256 chunk up to 2^23.1: any inexact
    fp32 accumulation would break the closed-form answer.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1208_4869_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ccg():
    from paper_1208_4869_gb300 import build as B
    B.build()
    from paper_1208_4869_gb300 import ccg as C
    return C


def colmajor(a):
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def product(ccg, A, X, fp64_tc=1):
    h = ccg.Handle()
    h.set_option(ccg.OPT_TC_FP64, fp64_tc)
    op = h.op_dense(torch.from_numpy(A).cuda())
    Y = colmajor(np.zeros(X.shape, np.complex128))
    h.block_matvec(op, colmajor(X), Y)
    torch.cuda.synchronize()
    return Y.cpu().numpy()


def exact_entry(A, X, i, c):
    """(A X)_ic as a pair of Fractions, every product and sum exact."""
    re = im = Fraction(0)
    for j in range(A.shape[1]):
        ar, ai = Fraction(float(A[i, j].real)), Fraction(float(A[i, j].imag))
        xr, xi = Fraction(float(X[j, c].real)), Fraction(float(X[j, c].imag))
        re += ar * xr - ai * xi
        im += ar * xi + ai * xr
    return re, im


def rmax(A, i):
    return max(np.abs(A[i].real).max(), np.abs(A[i].imag).max())


def cmax(X, c):
    return max(np.abs(X[:, c].real).max(), np.abs(X[:, c].imag).max())


def check_sampled(A, X, Y, entries, typical=True):
    K = 2 * A.shape[0]
    for i, c in entries:
        ex = exact_entry(A, X, i, c)
        mm = rmax(A, i) * cmax(X, c)
        for got, e in ((Y[i, c].real, ex[0]), (Y[i, c].imag, ex[1])):
            err = abs(Fraction(float(got)) - e)
            assert err <= Fraction(K * 2.0 ** -52 * mm) + abs(e) * Fraction(2.0 ** -52), (i, c, float(err))
            if typical:
                assert err <= Fraction(math.sqrt(K) * 2.0 ** -50 * mm) + abs(e) * Fraction(2.0 ** -52), \
                    (i, c, float(err), mm)


def sample(n, k, count, seed):
    rng = np.random.default_rng(seed)
    pts = {(0, 0), (n - 1, k - 1), (n - 1, 0), (0, k - 1)}
    count = min(count, n * k)
    while len(pts) < count:
        pts.add((int(rng.integers(n)), int(rng.integers(k))))
    return sorted(pts)


@pytest.mark.parametrize("n,k", [(4, 1), (132, 3), (256, 17), (1000, 37), (640, 64)])
def test_fp64_tc_ragged(ccg, n, k):
    """Ragged against the 128-row tile, the 32-column tile and K = 32 blocks,
    single and several K = 256 chunks (both tensor-memory buffers reused)."""
    A, _ = W.dense_system(n, 1.0, n)
    X = W.dense_rhs_block(n, k, seed=k)
    Y = product(ccg, A, X)
    check_sampled(A, X, Y, sample(n, k, 24, n + k))
    # every entry within the FP64 GEMM bound of numpy's own product
    ref = A @ X
    K = 2 * n
    mm = np.maximum(np.abs(A.real), np.abs(A.imag)).max(1)[:, None] * \
        np.maximum(np.abs(X.real), np.abs(X.imag)).max(0)[None, :]
    assert np.all(np.abs(Y - ref) <= 2 * K * 2.0 ** -53 * mm * 2 + 2.0 ** -51 * np.abs(ref))


def test_fp64_tc_scales(ccg):
    """Rows and columns scaled by powers of two from 2^-300 to 2^300, and
    non-power-of-two scales: the per-row and per-column exponents."""
    n, k = 384, 40
    rng = np.random.default_rng(7)
    A, _ = W.dense_system(n, 1.0, 5)
    X = W.dense_rhs_block(n, k, seed=8)
    A = A * np.ldexp(1.0, rng.integers(-300, 300, n))[:, None] * rng.uniform(0.5, 3.0, n)[:, None]
    X = X * np.ldexp(1.0, rng.integers(-300, 300, k))[None, :]
    Y = product(ccg, A, X)
    check_sampled(A, X, Y, sample(n, k, 32, 3))
    # rows of subnormal magnitude (row exponents near -1030)
    A2 = A.copy()
    A2[:4] = A[:4] / np.abs(A[:4]).max(1)[:, None] * 1e-310
    X2 = W.dense_rhs_block(n, k, seed=8)
    Y2 = product(ccg, A2, X2)
    check_sampled(A2, X2, Y2, [(i, c) for i in range(4) for c in (0, k - 1)], typical=False)


def test_fp64_tc_adversarial_digits(ccg):
    """Every entry a = v (1 - i), x = v (1 + i) with v's digits
    127, -63, 63, -63, ... (alternating at their bounds, so every digit-pair
    product of level l has the sign (-1)^l): each level's K = 256 chunk sum
    reaches up to 2^23.1 of the fp32 accumulator's 2^24 exact range.
    The answer is y = 2 n v^2 (real) for every entry."""
    D = [127] + [63 * (-1) ** t for t in range(1, 8)]
    v0 = sum(Fraction(d, 128 ** t) for t, d in enumerate(D))
    v = float(v0 / 128)                           # in (1/2, 1): exponent 0
    for n, k in ((1024, 32), (2048, 48)):
        A = np.full((n, n), complex(v, -v))
        X = np.full((n, k), complex(v, v))
        Y = product(ccg, A, X)
        exact = 2 * n * Fraction(v) ** 2
        bound = float(exact) * 2.0 ** -52
        assert np.all(np.abs(Y.real - float(exact)) <= bound), np.abs(Y.real - float(exact)).max()
        assert np.all(Y.imag == 0.0)


def test_fp64_tc_zero_and_nonfinite(ccg):
    n, k = 256, 5
    A, _ = W.dense_system(n, 1.0, 2)
    X = W.dense_rhs_block(n, k, seed=3)
    A[7, :] = 0.0
    X[:, 1] = 0.0
    Y = product(ccg, A, X)
    assert np.all(Y[7] == 0.0) and np.all(Y[:, 1] == 0.0)
    check_sampled(A, X, Y, [(0, 0), (8, 2), (n - 1, 4)])
    # a NaN in one column and an inf in one row poison exactly that column / row
    X2 = X.copy()
    X2[11, 3] = complex(np.nan, 0.0)
    A2 = A.copy()
    A2[20, 5] = complex(0.0, np.inf)
    Y2 = product(ccg, A2, X2)
    bad = np.zeros((n, k), bool)
    bad[:, 3] = True
    bad[20, :] = True
    assert np.all(np.isnan(Y2[bad].real))
    assert np.all(np.isfinite(Y2[~bad]))
    assert np.array_equal(Y2[~bad], Y[~bad])


def test_fp64_tc_matches_cuda_cores(ccg):
    """The CUDA-core FP64 product (option off) and the tensor-core one agree
    to the FP64 GEMM bound; both are close to the exact product."""
    n, k = 512, 24
    A, _ = W.dense_system(n, 1.0, 9)
    X = W.dense_rhs_block(n, k, seed=10)
    Yt = product(ccg, A, X, 1)
    Yc = product(ccg, A, X, 0)
    check_sampled(A, X, Yt, sample(n, k, 12, 1))
    check_sampled(A, X, Yc, sample(n, k, 12, 1), typical=False)
    assert np.abs(Yt - Yc).max() / np.abs(Yc).max() < 1e-14


def test_fp64_tc_full_size(ccg):
    """n = 8192, 256 right-hand sides (the multi-right-hand-side workload in
    complex128): sampled entries exact, every entry within the FP64 bound of
    numpy's product."""
    n, k = 8192, 256
    A, _ = W.dense_system(n, 3.0, 0)
    X = W.dense_rhs_block(n, k, seed=1)
    Y = product(ccg, A, X)
    check_sampled(A, X, Y, sample(n, k, 12, 5))
    ref = A @ X
    col = np.linalg.norm(Y - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert col.max() < 1e-13, col.max()


def test_batched_complex128_same_with_and_without_fp64_tc(ccg):
    """Batched complex128 BiCGSTAB with either product: the same converged
    solutions, and the same iteration counts within one."""
    n, k = 512, 16
    A, _ = W.dense_system(n, 1.0, 4)
    Y = W.dense_rhs_block(n, k, seed=6)
    out = []
    for mode in (0, 1):
        h = ccg.Handle()
        h.set_option(ccg.OPT_TC_FP64, mode)
        op = h.op_dense(torch.from_numpy(A).cuda())
        X = colmajor(np.zeros((n, k), np.complex128))
        st, iters, sts, rr = h.solve_batched("bicgstab", op, colmajor(Y), X, tol=1e-11, maxit=2000)
        assert st == 0 and np.all(rr <= 1e-11)
        Xh = X.cpu().numpy()
        assert np.all(np.linalg.norm(Y - A @ Xh, axis=0) / np.linalg.norm(Y, axis=0) <= 2e-11)
        out.append((Xh, iters))
    assert np.linalg.norm(out[0][0] - out[1][0]) / np.linalg.norm(out[0][0]) < 1e-9
    assert np.all(np.abs(out[0][1] - out[1][1]) <= 1)
