"""GPU parity of the batched (many right-hand sides) BiCGSTAB and its mixed-
precision refinement against the CPU oracle's single-right-hand-side
BiCGSTAB, column by column, through the C ABI.

Each column of a batched solve is the same method as a single solve of that
column (Sec. 1 problem, Sec. 2.1 method); only the block product's summation
order differs.  Tolerances as in the dense tests: complex128 iterates within
1e-9 relative; refined solutions to residual 1e-10 in complex128.
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


def colmajor(a, dtype=None):
    """(n, k) numpy array -> column-major CUDA tensor of shape (n, k)."""
    t = torch.from_numpy(np.ascontiguousarray(a.T if dtype is None else a.T.astype(dtype))).cuda()
    return t.t()


@pytest.mark.parametrize("k", [1, 7, 64])
def test_batched_iterates_match_single_solves(h, k):
    n = 300
    A, _ = W.dense_system(n, 0.8, 3)
    Y = W.dense_rhs_block(n, k, seed=4)
    op = h.op_dense(torch.from_numpy(A).cuda())
    oop = O.DenseOp(A)
    for it in (1, 4, 12):
        X = colmajor(np.zeros((n, k), np.complex128))
        st, iters, sts, rr = h.solve_batched("bicgstab", op, colmajor(Y), X, tol=0.0, maxit=it)
        Xh = X.cpu().numpy()
        for c in range(k):
            ref = O.solve(oop, "bicgstab", Y[:, c], tol=0.0, maxit=it)
            assert iters[c] == ref.iters == it
            assert np.linalg.norm(Xh[:, c] - ref.x) / np.linalg.norm(ref.x) < 1e-9, (c, it)


def test_batched_columns_stop_independently(h, ccg):
    """Columns of different difficulty: each stops at its own count, equal to
    its single-solve count; a zero column returns zero after 0 iterations."""
    n, k = 256, 9
    A, _ = W.dense_system(n, 2.0, 8)
    Y = W.dense_rhs_block(n, k, seed=5)
    Y[:, 3] = 0
    Y[:, 5] = A @ np.eye(n, dtype=np.complex128)[:, 7]       # an easy column
    op = h.op_dense(torch.from_numpy(A).cuda())
    oop = O.DenseOp(A)
    X = colmajor(W.dense_rhs_block(n, k, seed=6) * 0)
    st, iters, sts, rr = h.solve_batched("bicgstab", op, colmajor(Y), X, tol=1e-10, maxit=300)
    assert st == 0 and np.all(sts == 0)
    Xh = X.cpu().numpy()
    assert iters[3] == 0 and np.all(Xh[:, 3] == 0)
    for c in range(k):
        if c == 3:
            continue
        ref = O.solve(oop, "bicgstab", Y[:, c], tol=1e-10, maxit=300)
        assert iters[c] == ref.iters, c
        assert np.linalg.norm(Y[:, c] - A @ Xh[:, c]) / np.linalg.norm(Y[:, c]) <= 1e-10
        assert np.linalg.norm(Xh[:, c] - ref.x) / np.linalg.norm(ref.x) < 1e-9


def test_batched_fp32(h):
    n, k = 500, 16
    A, _ = W.dense_system(n, 3.0, 2)
    Y = W.dense_rhs_block(n, k, seed=2)
    op = h.op_dense(torch.from_numpy(A.astype(np.complex64)).cuda())
    X = colmajor(np.zeros((n, k), np.complex64))
    st, iters, sts, rr = h.solve_batched("bicgstab", op, colmajor(Y, np.complex64), X, tol=1e-6, maxit=200)
    assert st == 0
    Xh = X.cpu().numpy().astype(np.complex128)
    R = Y.astype(np.complex64).astype(np.complex128) - A.astype(np.complex64).astype(np.complex128) @ Xh
    assert np.all(np.linalg.norm(R, axis=0) / np.linalg.norm(Y, axis=0) < 3e-6)


@pytest.mark.parametrize("n,k", [(384, 40), (8192, 256)])
def test_batched_refined(h, n, k):
    """Mixed precision: complex64 batched BiCGSTAB inside complex128 block
    refinement; every column's complex128 residual <= 1e-10 and its solution
    equals the oracle's complex128 solution within the forward error.  At
    n = 8192, k = 256 this is the multi-right-hand-side workload."""
    shift = 3.0
    A, _ = W.dense_system(n, shift, 0)
    Y = W.dense_rhs_block(n, k, seed=1)
    Ad = torch.from_numpy(A).cuda()
    op64, op32 = h.op_dense(Ad), h.op_dense(Ad.to(torch.complex64))
    X = colmajor(np.zeros((n, k), np.complex128))
    st, outer, inner, sts, rr = h.solve_batched_refined("bicgstab", op64, op32, colmajor(Y), X, tol=1e-10)
    assert st == 0 and np.all(sts == 0) and np.all(rr <= 1e-10)
    Xh = X.cpu().numpy()
    R = Y - A @ Xh
    true = np.linalg.norm(R, axis=0) / np.linalg.norm(Y, axis=0)
    assert np.all(true <= 1e-10)
    assert np.allclose(true, rr, rtol=1e-3, atol=1e-13)
    oop = O.DenseOp(A)
    for c in sorted({0, k // 2, k - 1}):
        ref = O.solve(oop, "bicgstab", Y[:, c], tol=1e-12, maxit=500)
        assert np.linalg.norm(Xh[:, c] - ref.x) / np.linalg.norm(ref.x) < 1e-9, c
    assert np.all(outer >= 1) and np.all(inner >= outer)


def test_batched_argument_checks(h, ccg):
    n = 64
    A, _ = W.dense_system(n, 3.0, 1)
    op = h.op_dense(torch.from_numpy(A).cuda())
    X = colmajor(np.zeros((n, 4), np.complex128))
    Y = colmajor(W.dense_rhs_block(n, 4, seed=3))
    with pytest.raises(ccg.CcgError):
        h.solve_batched("qmr", op, Y, X)                     # only BiCGSTAB is batched
    big = colmajor(np.zeros((n, 257), np.complex128))
    with pytest.raises(ccg.CcgError):
        h.solve_batched("bicgstab", op, big, big)            # more than 256 columns
