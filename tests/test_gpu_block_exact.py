"""Exact-integer block products on the tensor cores (integer digit slices,
exact bf16 products, fp32 level sums, int64 combination) through the C ABI,
against exact rational references: FP64-accurate for complex128 (8 digits),
FP32-accurate for complex64 (4 digits).

The product Y = A X is the manual's `matvec` (Sec. 5) applied to a block of
right-hand sides.  complex128 bounds, with K = 2n real terms per entry:
  * rigorous: |y - exact| <= K 2^-52 max|a_i.| max|x_.c| + 2^-52 |exact|
    (8 seven-bit digits per operand keep 56 bits; the dropped digit pairs
    and remainders are below 2^-54.5 of 2^(e_i + f_c) per term, and
    2^(e_i + f_c) < 4 max|a_i.| max|x_.c|), the bound an FP64 GEMM obeys;
  * typical, for random signs: |y - exact| <= sqrt(K) 2^-50 max|a| max|x|
    + 2^-52 |exact|, far below what a lost digit level would leave;
  * the adversarial block whose digits all sit at their bounds with equal
    signs drives level sums of a K = 256 chunk up to 2^23.1: any inexact
    fp32 accumulation would break the closed-form answer.
complex64 (4 digits keep 28 bits; the dropped levels and remainders are
below 2^-27.4 of 2^(e_i + f_c) per term; one more rounding to float):
  * rigorous: |y - exact| <= K 2^-25 max|a_i.| max|x_.c| + 2^-23 |exact|;
  * typical: sqrt(K) 2^-22 max|a| max|x| + 2^-23 |exact|;
  * adversarial digits 127, -63, 63, -63 over K = 512 chunks: level sums up
    to 2^23.3.
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


def product(ccg, A, X, tc_exact=1):
    """Y = A X through ccg_block_matvec; complex64 with the split-bf16 path off."""
    h = ccg.Handle()
    h.set_option(ccg.OPT_TC_EXACT, tc_exact)
    h.set_option(ccg.OPT_TENSOR_CORES, 0)
    op = h.op_dense(torch.from_numpy(A).cuda())
    Y = colmajor(np.zeros(X.shape, A.dtype))
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
    c64 = A.dtype == np.complex64
    rig, typ, rel = (2.0 ** -25, 2.0 ** -22, 2.0 ** -23) if c64 else (2.0 ** -52, 2.0 ** -50, 2.0 ** -52)
    for i, c in entries:
        ex = exact_entry(A, X, i, c)
        mm = float(rmax(A, i)) * float(cmax(X, c))
        for got, e in ((Y[i, c].real, ex[0]), (Y[i, c].imag, ex[1])):
            err = abs(Fraction(float(got)) - e)
            assert err <= Fraction(K * rig * mm) + abs(e) * Fraction(rel), (i, c, float(err))
            if typical:
                assert err <= Fraction(math.sqrt(K) * typ * mm) + abs(e) * Fraction(rel), (i, c, float(err), mm)


def sample(n, k, count, seed):
    rng = np.random.default_rng(seed)
    pts = {(0, 0), (n - 1, k - 1), (n - 1, 0), (0, k - 1)}
    count = min(count, n * k)
    while len(pts) < count:
        pts.add((int(rng.integers(n)), int(rng.integers(k))))
    return sorted(pts)


@pytest.mark.parametrize("n,k", [(4, 1), (132, 3), (256, 17), (1000, 37), (640, 64)])
def test_fp64_exact_ragged(ccg, n, k):
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


def test_fp64_exact_scales(ccg):
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


def test_fp64_exact_adversarial_digits(ccg):
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


def test_fp64_exact_zero_and_nonfinite(ccg):
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


def test_fp64_exact_matches_cuda_cores(ccg):
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


def test_fp64_exact_full_size(ccg):
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


def test_batched_complex128_same_with_and_without_exact_products(ccg):
    """Batched complex128 BiCGSTAB with either product: the same converged
    solutions, and the same iteration counts within one."""
    n, k = 512, 16
    A, _ = W.dense_system(n, 1.0, 4)
    Y = W.dense_rhs_block(n, k, seed=6)
    out = []
    for mode in (0, 1):
        h = ccg.Handle()
        h.set_option(ccg.OPT_TC_EXACT, mode)
        op = h.op_dense(torch.from_numpy(A).cuda())
        X = colmajor(np.zeros((n, k), np.complex128))
        st, iters, sts, rr = h.solve_batched("bicgstab", op, colmajor(Y), X, tol=1e-11, maxit=2000)
        assert st == 0 and np.all(rr <= 1e-11)
        Xh = X.cpu().numpy()
        assert np.all(np.linalg.norm(Y - A @ Xh, axis=0) / np.linalg.norm(Y, axis=0) <= 2e-11)
        out.append((Xh, iters))
    assert np.linalg.norm(out[0][0] - out[1][0]) / np.linalg.norm(out[0][0]) < 1e-9
    assert np.all(np.abs(out[0][1] - out[1][1]) <= 1)


# ------------------------------------------------------------------ complex64 (4 digits)
@pytest.mark.parametrize("n,k", [(4, 1), (132, 3), (1000, 37), (640, 64)])
def test_fp32_exact_ragged(ccg, n, k):
    """Ragged against the 128-row tile, the 64-column tile and K = 32 blocks;
    several K = 512 chunks."""
    A, _ = W.dense_system(n, 1.0, n, dtype=np.complex64)
    X = W.dense_rhs_block(n, k, seed=k, dtype=np.complex64)
    Y = product(ccg, A, X)
    assert Y.dtype == np.complex64
    check_sampled(A, X, Y, sample(n, k, 24, n + k))


def test_fp32_exact_adversarial_digits(ccg):
    """a = v (1 - i), x = v (1 + i) with v's digits 127, -63, 63, -63 (as
    far as float keeps them): level sums of a K = 512 chunk up to 2^23.3;
    y = 2 n v^2 for every entry."""
    D = [127, -63, 63, -63]
    v0 = sum(Fraction(d, 128 ** t) for t, d in enumerate(D))
    v = float(np.float32(float(v0 / 128)))
    for n, k in ((1024, 64), (4096, 40)):
        A = np.full((n, n), complex(v, -v), np.complex64)
        X = np.full((n, k), complex(v, v), np.complex64)
        Y = product(ccg, A, X)
        exact = 2 * n * Fraction(v) ** 2
        assert np.all(np.abs(Y.real.astype(np.float64) - float(exact)) <= float(exact) * 2.0 ** -23)
        assert np.all(Y.imag == 0.0)


def test_fp32_exact_scales_and_nonfinite(ccg):
    n, k = 384, 40
    rng = np.random.default_rng(11)
    A, _ = W.dense_system(n, 1.0, 5, dtype=np.complex64)
    X = W.dense_rhs_block(n, k, seed=8, dtype=np.complex64)
    A = (A * np.ldexp(1.0, rng.integers(-60, 60, n))[:, None]).astype(np.complex64)
    X = (X * np.ldexp(1.0, rng.integers(-60, 60, k))[None, :]).astype(np.complex64)
    Y = product(ccg, A, X)
    check_sampled(A, X, Y, sample(n, k, 24, 3))
    X2 = X.copy()
    X2[11, 3] = complex(np.nan, 0.0)
    Y2 = product(ccg, A, X2)
    assert np.all(np.isnan(Y2[:, 3].real))
    keep = np.ones(k, bool)
    keep[3] = False
    assert np.array_equal(Y2[:, keep], Y[:, keep])


def test_fp32_exact_matches_cuda_cores(ccg):
    n, k = 512, 24
    A, _ = W.dense_system(n, 1.0, 9, dtype=np.complex64)
    X = W.dense_rhs_block(n, k, seed=10, dtype=np.complex64)
    Yt = product(ccg, A, X, 1)
    Yc = product(ccg, A, X, 0)
    check_sampled(A, X, Yt, sample(n, k, 12, 1))
    ref = A.astype(np.complex128) @ X.astype(np.complex128)
    et = np.abs(Yt - ref).max() / np.abs(ref).max()
    ec = np.abs(Yc - ref).max() / np.abs(ref).max()
    assert et < 1e-6 and ec < 2e-5, (et, ec)


def test_fp32_exact_full_size(ccg):
    """n = 8192, 256 right-hand sides in complex64: every column within
    FP32 accuracy of the complex128 product of the same data."""
    n, k = 8192, 256
    A, _ = W.dense_system(n, 3.0, 0, dtype=np.complex64)
    X = W.dense_rhs_block(n, k, seed=1, dtype=np.complex64)
    Y = product(ccg, A, X)
    check_sampled(A, X, Y, sample(n, k, 8, 5))
    ref = A.astype(np.complex128) @ X.astype(np.complex128)
    col = np.linalg.norm(Y - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert col.max() < 1e-6, col.max()


def test_refined_batched_same_with_and_without_exact_products(ccg):
    """Refined batched BiCGSTAB: the exact complex64 residual and the
    complex128 residuals on the tensor cores or on CUDA cores give the same
    converged solutions."""
    n, k = 640, 24
    A, _ = W.dense_system(n, 3.0, 0)
    Y = W.dense_rhs_block(n, k, seed=1)
    out = []
    for mode in (0, 1):
        h = ccg.Handle()
        h.set_option(ccg.OPT_TC_EXACT, mode)
        Ad = torch.from_numpy(A).cuda()
        op64, op32 = h.op_dense(Ad), h.op_dense(Ad.to(torch.complex64))
        X = colmajor(np.zeros((n, k), np.complex128))
        st, outer, inner, sts, rr = h.solve_batched_refined("bicgstab", op64, op32, colmajor(Y), X, tol=1e-10)
        assert st == 0 and np.all(rr <= 1e-10)
        Xh = X.cpu().numpy()
        assert np.all(np.linalg.norm(Y - A @ Xh, axis=0) / np.linalg.norm(Y, axis=0) <= 1e-10)
        out.append(Xh)
    assert np.linalg.norm(out[0] - out[1]) / np.linalg.norm(out[0]) < 1e-9


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
def test_exact_products_fallback_and_widest_block(ccg, dtype):
    """n not divisible by 4 falls back to the CUDA-core product (same
    accuracy class); n = 4 with the widest block, 256 right-hand sides."""
    for n, k in ((258, 5), (4, 256)):
        A, _ = W.dense_system(n, 1.0, n, dtype=dtype)
        X = W.dense_rhs_block(n, k, seed=3, dtype=dtype)
        Y = product(ccg, A, X)
        ref = A.astype(np.complex128) @ X.astype(np.complex128)
        e = np.abs(Y - ref).max() / np.abs(ref).max()
        assert e < (1e-13 if dtype == np.complex128 else 2e-5), (n, k, e)   # fp32 CUDA-core bound
