"""GPU parity at the full size of the dense single-right-hand-side workload.

n = 8192, A = (3 + 0.5 + 0.5i) I + G / sqrt(n), one complex-normal right-hand
side, x0 = 0: the configuration the benchmark times, with the same launch
geometry (row split of the A x sweep, row ranges of the A^H x and fused
A p + A^H q sweeps).  Each of the benchmark's three methods (Sec. 2.1
`bicgstab`, `cgnr`, `qmr`) is solved

  * in complex128: the whole solve against the oracle's -- equal iteration
    counts, residual history within 1e-8 relative (above an absolute floor
    of 1e-13 ||y||), x within 1e-9;
  * with complex64 inner solves inside complex128 refinement (the
    benchmark's headline path): final true residual <= 1e-10, x within 1e-9
    of the oracle's complex128 solution (the forward error a 1e-10 residual
    allows at cond(A) ~ 2.3), and the number of corrections within one of
    the oracle's own refinement;
  * in complex64 alone to 1e-6 (the plain single-precision path), the true
    residual taken by the oracle in double.

The oracle's solves (about 1-5 s each on one host core) are computed once
per method and shared by the three paths.
"""
import numpy as np
import pytest

import oracle as O
from paper_1208_4869_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = W.DENSE_LARGE["n"]
METHODS = ["bicgstab", "cgnr", "qmr"]


@pytest.fixture(scope="module")
def ccg():
    from paper_1208_4869_gb300 import build as B
    B.build()
    from paper_1208_4869_gb300 import ccg as C
    return C


@pytest.fixture(scope="module")
def h(ccg):
    return ccg.Handle()


@pytest.fixture(scope="module")
def system():
    return W.dense_system(**W.DENSE_LARGE)


@pytest.fixture(scope="module")
def dev_ops(h, system):
    A, _ = system
    Ad = torch.from_numpy(A).cuda()
    A32 = Ad.to(torch.complex64)
    return h.op_dense(Ad), h.op_dense(A32), (Ad, A32)


_oracle_cache = {}


def oracle_solution(system, method):
    if method not in _oracle_cache:
        A, y = system
        _oracle_cache[method] = O.solve(O.DenseOp(A), method, y, tol=1e-10, maxit=300)
    return _oracle_cache[method]


def relres(A, x, y):
    return np.linalg.norm(y - A @ x) / np.linalg.norm(y)


@pytest.mark.parametrize("method", METHODS)
def test_full_size_fp64_matches_oracle(h, system, dev_ops, method):
    A, y = system
    op64, _, _ = dev_ops
    ref = oracle_solution(system, method)
    assert ref.status == O.OK
    xd = torch.zeros(N, dtype=torch.complex128, device="cuda")
    st, info, hist = h.solve(method, op64, torch.from_numpy(y).cuda(), xd, tol=1e-10, maxit=300)
    assert st == 0 and info["iters"] == ref.iters
    # The recurrence residuals (r -= alpha w, r -= s, r = s - omega t) keep
    # the rounding of every earlier update at the scale of ||r_0|| = ||y||,
    # so late entries are compared on that scale: rtol 1e-8, plus an absolute
    # floor of 1e-13 ||y|| (about sqrt(n) eps: matrix-vector sums in another
    # order than the oracle's).
    assert np.allclose(hist, ref.hist, rtol=1e-8, atol=1e-13)
    x = xd.cpu().numpy()
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) < 1e-9
    assert info["relres"] <= 1e-10
    # the true residual, recomputed on the device and by numpy
    assert abs(info["true_relres"] - relres(A, x, y)) <= 1e-13
    # the recurrence residual the solve stopped on has not drifted from it
    assert abs(info["true_relres"] - info["relres"]) <= 1e-13


@pytest.mark.parametrize("method", METHODS)
def test_full_size_refined_matches_oracle(h, system, dev_ops, method):
    A, y = system
    op64, op32, _ = dev_ops
    ref = oracle_solution(system, method)
    xd = torch.zeros(N, dtype=torch.complex128, device="cuda")
    st, info, hist, inner = h.solve_refined(method, op64, op32, torch.from_numpy(y).cuda(), xd, tol=1e-10,
                                            max_outer=30, inner_tol=1e-5, inner_maxit=200)
    x = xd.cpu().numpy()
    assert st == 0
    assert info["true_relres"] <= 1e-10 and relres(A, x, y) <= 1e-10
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) < 1e-9
    assert hist[-1] <= 1e-10 and np.all(np.diff(hist) < 0)
    _, outer, ost, oinner, _ = O.refine(O.DenseOp(A), O.DenseOp(A.astype(np.complex64)), method, y, tol=1e-10,
                                        max_outer=30, inner_tol=1e-5, inner_maxit=200)
    assert ost == O.OK
    assert abs(info["iters"] - outer) <= 1
    assert 0 < inner <= 200 * info["iters"]


@pytest.mark.parametrize("method", METHODS)
def test_full_size_fp32_reaches_1e6(h, system, dev_ops, method):
    A, y = system
    _, op32, _ = dev_ops
    xd = torch.zeros(N, dtype=torch.complex64, device="cuda")
    st, info, _ = h.solve(method, op32, torch.from_numpy(y.astype(np.complex64)).cuda(), xd, tol=1e-6, maxit=300)
    assert st == 0 and info["relres"] <= 1e-6
    x = xd.cpu().numpy().astype(np.complex128)
    assert relres(A.astype(np.complex64).astype(np.complex128), x, y.astype(np.complex64)) < 3e-6
