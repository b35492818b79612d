"""The OpenMP build of the oracle (the benchmark's all-core CPU baseline)
computes exactly what the serial oracle computes: its threads only take
independent output elements of the dense products, so every sum keeps its
order and the results are bit-identical."""
import numpy as np
import pytest

import oracle as O
from paper_1208_4869_gb300 import workloads as W


@pytest.fixture(scope="module")
def have_omp():
    try:
        O.lib(parallel=True)
    except Exception as e:  # a compiler without OpenMP support
        pytest.skip("no OpenMP build: %s" % e)


def test_serial_build_is_single_threaded():
    assert O.threads(parallel=False) == 1


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
@pytest.mark.parametrize("n", [1, 5, 255, 257, 600])
def test_products_bit_identical(have_omp, dtype, n):
    A, _ = W.dense_system(n, 2.0, n, dtype=dtype)
    x = W.random_vector(n, 7, dtype)
    s, p = O.DenseOp(A), O.DenseOp(A, parallel=True)
    for trans in (False, True):
        assert np.array_equal(s.matvec(x, trans), p.matvec(x, trans))
    # and against the definition, independently of either build
    ref = A.astype(np.complex128) @ x.astype(np.complex128)
    tol = 1e-12 if dtype == np.complex128 else 1e-5
    assert np.abs(s.matvec(x) - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("method", ["bicgstab", "cgnr", "qmr"])
def test_solves_and_refinement_bit_identical(have_omp, method):
    A, y = W.dense_system(300, 3.0, 4)
    r1 = O.solve(O.DenseOp(A), method, y, tol=1e-10, maxit=200)
    r2 = O.solve(O.DenseOp(A, parallel=True), method, y, tol=1e-10, maxit=200)
    assert r1.iters == r2.iters and np.array_equal(r1.x, r2.x) and np.array_equal(r1.hist, r2.hist)
    a = O.refine(O.DenseOp(A), O.DenseOp(A.astype(np.complex64)), method, y, tol=1e-10)
    b = O.refine(O.DenseOp(A, parallel=True), O.DenseOp(A.astype(np.complex64), parallel=True), method, y,
                 tol=1e-10)
    assert a[1:4] == b[1:4] and np.array_equal(a[0], b[0])
